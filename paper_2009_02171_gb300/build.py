"""In-tree build of libfv.so (CUDA, sm_103a) from csrc/*.cu.

Each translation unit is compiled in parallel with
`nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo -Xcompiler -fPIC`
and the objects are linked into paper_2009_02171_gb300/libfv.so.  No machine-
specific host flags are used, so the same sources build on x86_64 and aarch64.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
OUT = os.path.join(HERE, 'libfv.so')
BUILD = os.path.join(HERE, '_build')
NVCC = os.environ.get('NVCC', 'nvcc')
FLAGS = ['-gencode', 'arch=compute_103a,code=sm_103a', '-O3', '-lineinfo', '-std=c++17',
         '-Xcompiler', '-fPIC', '-Xptxas', '-v']


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith('.cu'))


def _compile(src):
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + '.o')
    cmd = [NVCC, *FLAGS, '-c', src, '-o', obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    with open(obj + '.log', 'w') as f:
        f.write(' '.join(cmd) + '\n' + p.stdout + p.stderr)
    if p.returncode != 0:
        raise RuntimeError('nvcc failed on %s:\n%s' % (src, p.stderr[-4000:]))
    return obj


def build(force=False):
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(('.h', '.cuh'))]
    deps += [os.path.join(HERE, '..', 'include', h) for h in ('fv.h', 'fv_net.h')]
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) > max(os.path.getmtime(d) for d in deps):
        return OUT
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(_compile, srcs))
    cmd = [NVCC, '-shared', '-gencode', 'arch=compute_103a,code=sm_103a', *objs, '-o', OUT + '.tmp', '-lcudart']
    subprocess.run(cmd, check=True)
    os.replace(OUT + '.tmp', OUT)
    return OUT


if __name__ == '__main__':
    print(build(force='--force' in sys.argv))
