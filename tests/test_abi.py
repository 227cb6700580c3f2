"""The C-ABI library loads and exports every symbol include/fv.h and include/fv_net.h declare (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, 'paper_2009_02171_gb300', 'libfv.so')


def _declared():
    src = ''.join(open(os.path.join(ROOT, 'include', h)).read() for h in ('fv.h', 'fv_net.h'))
    return sorted(set(re.findall(r'^\s*(?:fv_status|const char\*)\s+(fv_\w+)\s*\(', src, re.M)))


@pytest.fixture(scope='module')
def lib():
    if not os.path.exists(LIB):
        from paper_2009_02171_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ('fv_build_grid', 'fv_assemble_system', 'fv_apply_op', 'fv_precond_apply', 'fv_gmres_solve',
              'fv_time_step', 'fv_last_error', 'fv_net_create', 'fv_net_forward', 'fv_net_loss_grad',
              'fv_net_train', 'fv_pc_set_learned'):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_signatures_cover_the_header():
    src = open(os.path.join(ROOT, 'paper_2009_02171_gb300', 'fv.py')).read()
    for n in _declared():
        assert "'%s'" % n in src, n
