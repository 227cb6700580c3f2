// Learned coarse correction: a panel-wise 3-D convolutional U-Net on the coarse
// grid of the two-level preconditioner (declared in include/fv_net.h; not in the
// paper, it stands in for the coarse solve of eqn:coarsesolve).
//
// Data layout: activations and gradients are BF16, channels last, one voxel per
// coarse cell: [panel][k][j][i][channel] with panel = sample * 6 + cubed-sphere
// panel.  A convolution is an implicit GEMM (M = voxels, N = output channels,
// K = 27 taps x input channels) on the tensor cores (mma.sync m16n8k16, BF16 x
// BF16 -> FP32): one CTA computes a 4 x 4 x 8 brick of output voxels from a
// (6 x 6 x 10)-voxel halo of its input staged in shared memory (channel stride
// padded by 8 so ldmatrix rows fall in distinct banks).  The backward data pass
// is the same kernel with flipped, transposed weights; the weight gradient is a
// GEMM over voxels (M = input channels, N = output channels) split over
// (tap, voxel range) CTAs with FP32 atomics into the master gradient.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/fv_net.h"
#include "fv_internal.h"

namespace fv {
namespace {

using bf16 = __nv_bfloat16;

constexpr int BZ = 4, BY = 4, BX = 8;  // output brick of one convolution CTA (128 voxels, 4 warps)
constexpr int HY = BY + 2, HX = BX + 2, HV = (BZ + 2) * HY * HX;
constexpr int CONV_THREADS = 128;
constexpr int WK = 64;                 // voxels per weight-gradient chunk
constexpr int RED_THREADS = 256;

enum { EPI_RELU = 0, EPI_RAW = 1, EPI_MASK = 2, EPI_FINAL = 3 };

struct ConvArgs {
  const bf16* s0;     // full-resolution input, c0 channels
  const bf16* s1;     // half-resolution input read through nearest upsampling, c1 channels (or null)
  const bf16* w;      // [27][coutN][cin], tap = dz * 9 + dy * 3 + dx, input voxel = output + (dz, dy, dx) - 1
  const float* bias;  // [cout] (RELU, FINAL)
  const bf16* mask;   // [voxel][cout] (MASK): output kept where mask > 0
  bf16* out;          // [voxel][cout]
  float* y;           // [voxel][cout] FP32 (FINAL)
  int c0, c1, cin, coutN, cout;
  int P, Z, Y, X;
  int mode;
};

__device__ __forceinline__ void ldsm4(uint32_t addr, uint32_t* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldsm4t(uint32_t addr, uint32_t* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Load one 16-byte channel group q (8 channels) of the (possibly concatenated)
// input at voxel (p, z, y, x); zero outside the panel.
__device__ __forceinline__ uint4 load_in(const bf16* s0, int c0, const bf16* s1, int c1, int q, int p, int z,
                                         int y, int x, int Z, int Y, int X) {
  if (z < 0 || z >= Z || y < 0 || y >= Y || x < 0 || x >= X) return make_uint4(0, 0, 0, 0);
  if (q * 8 < c0) return *reinterpret_cast<const uint4*>(s0 + ((((long long)p * Z + z) * Y + y) * X + x) * c0 + q * 8);
  const int Zh = Z >> 1, Yh = Y >> 1, Xh = X >> 1;
  return *reinterpret_cast<const uint4*>(
      s1 + ((((long long)p * Zh + (z >> 1)) * Yh + (y >> 1)) * Xh + (x >> 1)) * c1 + (q * 8 - c0));
}

template <int NT>
__global__ void __launch_bounds__(CONV_THREADS) conv_kernel(ConvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16* hs = reinterpret_cast<bf16*>(smem_raw);
  const int cs = a.cin + 8;
  const int nbx = (a.X + BX - 1) / BX, nby = (a.Y + BY - 1) / BY, nbz = (a.Z + BZ - 1) / BZ;
  int blk = blockIdx.x;
  const int bx = blk % nbx;
  blk /= nbx;
  const int by = blk % nby;
  blk /= nby;
  const int bz = blk % nbz;
  const int p = blk / nbz;
  const int x0 = bx * BX, y0 = by * BY, z0 = bz * BZ;

  const int qn = a.cin >> 3;
  for (int it = threadIdx.x; it < HV * qn; it += CONV_THREADS) {
    const int hv = it / qn, q = it - hv * qn;
    const int hx = hv % HX, hy = (hv / HX) % HY, hz = hv / (HX * HY);
    const uint4 v = load_in(a.s0, a.c0, a.s1, a.c1, q, p, z0 - 1 + hz, y0 - 1 + hy, x0 - 1 + hx, a.Z, a.Y, a.X);
    *reinterpret_cast<uint4*>(hs + hv * cs + q * 8) = v;
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;

  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(hs);
  // A rows: lane & 15 = row of the m16 tile (y offset row >> 3, x offset row & 7), lane >> 4 = k half
  const int r = lane & 15, kh = lane >> 4;
  int hv0[2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) hv0[mt] = (warp * HY + 2 * mt + (r >> 3)) * HX + (r & 7);
  const int nq = lane >> 2, kq = (lane & 3) * 2;
  for (int tap = 0; tap < 27; ++tap) {
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    const int toff = (dz * HY + dy) * HX + dx;
    const bf16* wt = a.w + (size_t)tap * a.coutN * a.cin + (size_t)nq * a.cin + kq;
    for (int kc = 0; kc < a.cin; kc += 16) {
      uint32_t af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) ldsm4(sbase + (uint32_t)(((hv0[mt] + toff) * cs + kc + kh * 8) * 2), af[mt]);
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const bf16* wp = wt + (size_t)nt * 8 * a.cin + kc;
        const uint32_t b0 = __ldg(reinterpret_cast<const unsigned int*>(wp));
        const uint32_t b1 = __ldg(reinterpret_cast<const unsigned int*>(wp + 8));
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma16816(acc[mt][nt], af[mt], b0, b1);
      }
    }
  }

  // epilogue: accumulator e of tile (mt, nt): row (lane >> 2) + 8 (e >> 1), column nt*8 + (lane & 3)*2 + (e & 1)
  const int z = z0 + warp;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = (lane >> 2) + 8 * h;
      const int y = y0 + 2 * mt + (row >> 3), x = x0 + (row & 7);
      if (z >= a.Z || y >= a.Y || x >= a.X) continue;
      const long long v = (((long long)p * a.Z + z) * a.Y + y) * a.X + x;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int col = nt * 8 + (lane & 3) * 2;
        float u0 = acc[mt][nt][2 * h], u1 = acc[mt][nt][2 * h + 1];
        if (a.mode == EPI_FINAL) {
          if (col < a.cout) a.y[v * a.cout + col] = u0 + a.bias[col];
          if (col + 1 < a.cout) a.y[v * a.cout + col + 1] = u1 + a.bias[col + 1];
          continue;
        }
        if (col >= a.cout) continue;
        if (a.mode == EPI_RELU) {
          u0 = fmaxf(u0 + a.bias[col], 0.f);
          u1 = fmaxf(u1 + a.bias[col + 1], 0.f);
        } else if (a.mode == EPI_MASK) {
          const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(a.mask + v * a.cout + col);
          if (!(__bfloat162float(m.x) > 0.f)) u0 = 0.f;
          if (!(__bfloat162float(m.y) > 0.f)) u1 = 0.f;
        }
        *reinterpret_cast<__nv_bfloat162*>(a.out + v * a.cout + col) = __floats2bfloat162_rn(u0, u1);
      }
    }
}

// Weight gradient of one convolution: gw[co][ci][tap] += sum over voxels v of
// in[v + tap offset][ci] * g[v][co].  CTA (chunk group, tap); warp pairs
// (16 input channels) x (16 output channels) accumulate over WK-voxel chunks.
struct WGradArgs {
  const bf16* s0;
  const bf16* s1;
  const bf16* g;
  float* gw;
  int c0, c1, cin, gc, ci, co;
  int P, Z, Y, X;
  long long chunks_per_cta;
};

constexpr int WG_PAIRS = 4;  // (16 x 16) output tiles per warp: cin/16 * gc/16 <= 16

__global__ void __launch_bounds__(CONV_THREADS) wgrad_kernel(WGradArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int xsn = a.cin + 8, gsn = a.gc + 8;
  bf16* xs = reinterpret_cast<bf16*>(smem_raw);
  bf16* gs = xs + WK * xsn;
  const int tap = blockIdx.y;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const long long V = (long long)a.P * a.Z * a.Y * a.X;
  const long long nchunk = (V + WK - 1) / WK;
  const long long c_begin = blockIdx.x * a.chunks_per_cta;
  const long long c_end = nchunk < c_begin + a.chunks_per_cta ? nchunk : c_begin + a.chunks_per_cta;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n16 = a.gc >> 4, pairs = (a.cin >> 4) * n16;
  float acc[WG_PAIRS][2][4];
#pragma unroll
  for (int i = 0; i < WG_PAIRS; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][h][e] = 0.f;
  const uint32_t xbase = (uint32_t)__cvta_generic_to_shared(xs), gbase = (uint32_t)__cvta_generic_to_shared(gs);
  const int q = lane >> 3, i8 = lane & 7;
  const int qx = a.cin >> 3, qg = a.gc >> 3;
  for (long long ch = c_begin; ch < c_end; ++ch) {
    __syncthreads();
    for (int it = threadIdx.x; it < WK * qx; it += CONV_THREADS) {
      const int k = it / qx, qq = it - k * qx;
      const long long v = ch * WK + k;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (v < V) {
        long long t = v;
        const int x = (int)(t % a.X);
        t /= a.X;
        const int y = (int)(t % a.Y);
        t /= a.Y;
        const int z = (int)(t % a.Z);
        const int p = (int)(t / a.Z);
        val = load_in(a.s0, a.c0, a.s1, a.c1, qq, p, z + dz, y + dy, x + dx, a.Z, a.Y, a.X);
      }
      *reinterpret_cast<uint4*>(xs + k * xsn + qq * 8) = val;
    }
    for (int it = threadIdx.x; it < WK * qg; it += CONV_THREADS) {
      const int k = it / qg, qq = it - k * qg;
      const long long v = ch * WK + k;
      const uint4 val = v < V ? *reinterpret_cast<const uint4*>(a.g + v * a.gc + qq * 8) : make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(gs + k * gsn + qq * 8) = val;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < WK / 16; ++kk) {
#pragma unroll
      for (int i = 0; i < WG_PAIRS; ++i) {
        const int pr = warp + 4 * i;
        if (pr >= pairs) continue;
        const int mt = pr / n16, nt = pr - mt * n16;
        uint32_t af[4], bf[4];
        // A = in^T (m = input channel, k = voxel): matrix q covers voxels (q >> 1) * 8, channels (q & 1) * 8
        ldsm4t(xbase + (uint32_t)(((kk * 16 + (q >> 1) * 8 + i8) * xsn + mt * 16 + (q & 1) * 8) * 2), af);
        // B = g (k = voxel, n = output channel): matrix q covers voxels (q & 1) * 8, channels (q >> 1) * 8
        ldsm4t(gbase + (uint32_t)(((kk * 16 + (q & 1) * 8 + i8) * gsn + nt * 16 + (q >> 1) * 8) * 2), bf);
        mma16816(acc[i][0], af, bf[0], bf[1]);
        mma16816(acc[i][1], af, bf[2], bf[3]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < WG_PAIRS; ++i) {
    const int pr = warp + 4 * i;
    if (pr >= pairs) continue;
    const int mt = pr / n16, nt = pr - mt * n16;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = mt * 16 + (lane >> 2) + 8 * (e >> 1);
        const int n = nt * 16 + h * 8 + (lane & 3) * 2 + (e & 1);
        if (m < a.ci && n < a.co) atomicAdd(a.gw + ((long long)n * a.ci + m) * 27 + (blockIdx.y), acc[i][h][e]);
      }
  }
}

// bias gradient: gb[c] += sum over voxels of g[v][c]
__global__ void bgrad_kernel(const bf16* __restrict__ g, int gc, int co, long long V, float* gb) {
  __shared__ float part[RED_THREADS];
  const int rows = RED_THREADS / gc;  // gc divides RED_THREADS (16, 32, 64)
  const int c = threadIdx.x % gc, r = threadIdx.x / gc;
  float s = 0.f;
  if (r < rows)
    for (long long v = (long long)blockIdx.x * rows + r; v < V; v += (long long)gridDim.x * rows)
      s += __bfloat162float(g[v * gc + c]);
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < gc) {
    float t = 0.f;
    for (int k = 0; k < rows; ++k) t += part[k * gc + threadIdx.x];
    if (threadIdx.x < co) atomicAdd(gb + threadIdx.x, t);
  }
}

// 2x2x2 mean pooling (forward) of a [voxel][C] BF16 tensor
__global__ void pool_kernel(const bf16* __restrict__ a, bf16* __restrict__ p, int C, int P, int Z, int Y, int X) {
  const int Zh = Z / 2, Yh = Y / 2, Xh = X / 2, qn = C / 8;
  const long long n = (long long)P * Zh * Yh * Xh * qn;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < n; it += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(it % qn);
    long long t = it / qn;
    const int x = (int)(t % Xh);
    t /= Xh;
    const int y = (int)(t % Yh);
    t /= Yh;
    const int z = (int)(t % Zh);
    const int pp = (int)(t / Zh);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = 0; c < 8; ++c) {
      const long long v = (((long long)pp * Z + 2 * z + (c >> 2)) * Y + 2 * y + ((c >> 1) & 1)) * X + 2 * x + (c & 1);
      const uint4 u = *reinterpret_cast<const uint4*>(a + v * C + q * 8);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
      for (int k = 0; k < 4; ++k) {
        s[2 * k] += __bfloat162float(h[k].x);
        s[2 * k + 1] += __bfloat162float(h[k].y);
      }
    }
    uint4 o;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&o);
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(0.125f * s[2 * k], 0.125f * s[2 * k + 1]);
    *reinterpret_cast<uint4*>(p + (it / qn) * C + q * 8) = o;
  }
}

// backward through upsample + concat + ReLU of a4:
// g4[pv][c] = (sum over the 8 children of gcat[child][C + c]) * (a4[pv][c] > 0),  c < 2C
__global__ void g4_kernel(const bf16* __restrict__ gcat, const bf16* __restrict__ a4, bf16* __restrict__ g4, int C,
                          int P, int Z, int Y, int X) {
  const int Zh = Z / 2, Yh = Y / 2, Xh = X / 2, C2 = 2 * C;
  const long long n = (long long)P * Zh * Yh * Xh * C2;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < n; it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % C2);
    long long t = it / C2;
    const int x = (int)(t % Xh);
    t /= Xh;
    const int y = (int)(t % Yh);
    t /= Yh;
    const int z = (int)(t % Zh);
    const int pp = (int)(t / Zh);
    float s = 0.f;
    for (int k = 0; k < 8; ++k) {
      const long long v = (((long long)pp * Z + 2 * z + (k >> 2)) * Y + 2 * y + ((k >> 1) & 1)) * X + 2 * x + (k & 1);
      s += __bfloat162float(gcat[v * 3 * C + C + c]);
    }
    g4[it] = __float2bfloat16_rn(__bfloat162float(a4[it]) > 0.f ? s : 0.f);
  }
}

// backward through the skip path and the pooling into a2:
// g2[v][c] = (gcat[v][c] + gp[parent][c] / 8) * (a2[v][c] > 0),  c < C
__global__ void g2_kernel(const bf16* __restrict__ gcat, const bf16* __restrict__ gp, const bf16* __restrict__ a2,
                          bf16* __restrict__ g2, int C, int P, int Z, int Y, int X) {
  const long long n = (long long)P * Z * Y * X * C;
  const int Zh = Z / 2, Yh = Y / 2, Xh = X / 2;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < n; it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % C);
    long long t = it / C;
    const long long v = t;
    const int x = (int)(t % X);
    t /= X;
    const int y = (int)(t % Y);
    t /= Y;
    const int z = (int)(t % Z);
    const int pp = (int)(t / Z);
    const long long pv = (((long long)pp * Zh + z / 2) * Yh + y / 2) * Xh + x / 2;
    const float s = __bfloat162float(gcat[v * 3 * C + c]) + 0.125f * __bfloat162float(gp[pv * C + c]);
    g2[it] = __float2bfloat16_rn(__bfloat162float(a2[it]) > 0.f ? s : 0.f);
  }
}

// per-sample sum of squares of a coarse vector batch (sample b: 2 * V1 values)
template <class T>
__global__ void sumsq_kernel(const T* __restrict__ r, long long n1, double* ss) {
  __shared__ double part[RED_THREADS];
  const T* rb = r + blockIdx.y * n1;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)RED_THREADS + threadIdx.x; i < n1; i += (long long)gridDim.x * RED_THREADS) {
    const double v = (double)rb[i];
    s += v * v;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(ss + blockIdx.y, part[0]);
}

// x[v][0..15] = (r_P, r_Pb) / s, zero channels 2..15
template <class T>
__global__ void pack_kernel(const T* __restrict__ r, const double* __restrict__ ss, long long V1, int nb,
                            bf16* __restrict__ x) {
  const long long n = V1 * nb;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const long long b = v / V1, vl = v - b * V1;
    const double s2 = ss[b];
    const float inv = s2 > 0.0 ? (float)(1.0 / sqrt(s2)) : 0.f;
    uint4 o[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(o);
    h[0] = __floats2bfloat162_rn((float)r[b * 2 * V1 + vl] * inv, (float)r[b * 2 * V1 + V1 + vl] * inv);
    uint4* dst = reinterpret_cast<uint4*>(x + v * 16);
    dst[0] = o[0];
    dst[1] = o[1];
  }
}

// e[b][c][vl] = s_b * y[v][c]
template <class T>
__global__ void unpack_kernel(const float* __restrict__ y, const double* __restrict__ ss, long long V1, int nb,
                              T* __restrict__ e) {
  const long long n = V1 * nb;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const long long b = v / V1, vl = v - b * V1;
    const double s = sqrt(ss[b]);
    e[b * 2 * V1 + vl] = (T)(s * (double)y[2 * v]);
    e[b * 2 * V1 + V1 + vl] = (T)(s * (double)y[2 * v + 1]);
  }
}

// loss = sum over entries of (y - e/s)^2 (accumulated), gy = 2 (y - e/s) / ntot (channels 0, 1 of 16)
__global__ void loss_kernel(const float* __restrict__ y, const double* __restrict__ e, const double* __restrict__ ss,
                            long long V1, int nb, double inv_ntot, bf16* __restrict__ gy, double* loss) {
  __shared__ double part[RED_THREADS];
  const long long n = V1 * nb;
  double acc = 0.0;
  for (long long v = blockIdx.x * (long long)RED_THREADS + threadIdx.x; v < n; v += (long long)gridDim.x * RED_THREADS) {
    const long long b = v / V1, vl = v - b * V1;
    const double s2 = ss[b];
    const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
    const double d0 = (double)y[2 * v] - e[b * 2 * V1 + vl] * inv;
    const double d1 = (double)y[2 * v + 1] - e[b * 2 * V1 + V1 + vl] * inv;
    acc += d0 * d0 + d1 * d1;
    uint4 o[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
    reinterpret_cast<__nv_bfloat162*>(o)[0] =
        __floats2bfloat162_rn((float)(2.0 * d0 * inv_ntot), (float)(2.0 * d1 * inv_ntot));
    uint4* dst = reinterpret_cast<uint4*>(gy + v * 16);
    dst[0] = o[0];
    dst[1] = o[1];
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, part[0]);
}

// Adam (Kingma & Ba 2015, Algorithm 1) on FP32 masters; c1 = 1 - beta1^t, c2 = 1 - beta2^t
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 copies of one layer's master weights W[co][ci][27]:
// wf[tap][n = co][k = ci] (forward) and wb[tap][n = ci][k = co] = W[co][ci][26 - tap] (backward data)
__global__ void packw_kernel(const float* __restrict__ W, int ci, int co, int ciK, int coN, int ciN, int coK,
                             bf16* __restrict__ wf, bf16* __restrict__ wb) {
  const int nf = 27 * coN * ciK, nbk = wb ? 27 * ciN * coK : 0;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nf + nbk; it += gridDim.x * blockDim.x) {
    if (it < nf) {
      const int k = it % ciK, n = (it / ciK) % coN, tap = it / (ciK * coN);
      wf[it] = __float2bfloat16_rn(n < co && k < ci ? W[((long long)n * ci + k) * 27 + tap] : 0.f);
    } else {
      const int j = it - nf;
      const int k = j % coK, n = (j / coK) % ciN, tap = j / (coK * ciN);
      wb[j] = __float2bfloat16_rn(n < ci && k < co ? W[((long long)k * ci + n) * 27 + (26 - tap)] : 0.f);
    }
  }
}

int r16(int c) { return (c + 15) / 16 * 16; }
int r8(int c) { return (c + 7) / 8 * 8; }
int gridsz(long long n, int threads) { return (int)std::max(1LL, std::min((n + threads - 1) / threads, 304LL * 8)); }

}  // namespace

struct NetLayer {
  int ci, co;            // logical channels
  int ciK, coN, ciN, coK;  // padded: forward input (x16), forward output tile (x8), backward output, backward input
  long long woff, boff;  // offsets of W and b in the flat parameters
  bf16 *wf = nullptr, *wb = nullptr;
};

}  // namespace fv

struct fv_net {
  int C = 0, Ns = 0, Nr = 0, nbmax = 0;
  int Z = 0, Y = 0, X = 0;
  long long V1 = 0;       // coarse cells of one sample (6 Ns^2 Nr)
  long long nparam = 0;
  fv::NetLayer L[6];
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 masters, gradient, Adam moments
  long long t = 0;        // Adam step counter
  double* ss = nullptr;   // [nbmax] per-sample sum of squares
  double* loss = nullptr; // [1]
  // activations (BF16, channels last)
  fv::bf16 *x = nullptr, *a1 = nullptr, *a2 = nullptr, *p = nullptr, *a3 = nullptr, *a4 = nullptr, *a5 = nullptr;
  float* y = nullptr;
  // gradients (allocated on first training call)
  fv::bf16 *gy = nullptr, *g5 = nullptr, *gcat = nullptr, *g4 = nullptr, *g3 = nullptr, *gp = nullptr,
           *g2 = nullptr, *g1 = nullptr;
  double *rb = nullptr, *eb = nullptr;  // training batch staging
  std::vector<void*> allocs;
};

namespace fv {
namespace {

template <class T>
fv_status nalloc(fv_net* n, T** p, size_t count) {
  if (cudaMalloc(p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess)
    return set_error("fv_net: device allocation failed"), FV_ENOMEM;
  n->allocs.push_back(*p);
  return FV_OK;
}

template <int NT>
fv_status conv_launch_nt(const ConvArgs& a, int blocks, size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    FV_CUDA(cudaFuncSetAttribute(conv_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, HV * (96 + 8) * 2));
    attr = true;
  }
  conv_kernel<NT><<<blocks, CONV_THREADS, smem, st>>>(a);
  return FV_OK;
}

fv_status conv(const ConvArgs& a, cudaStream_t st) {
  const int blocks = a.P * ((a.Z + BZ - 1) / BZ) * ((a.Y + BY - 1) / BY) * ((a.X + BX - 1) / BX);
  const size_t smem = (size_t)HV * (a.cin + 8) * 2;
  if (a.cin % 16 || a.c0 % 8 || a.cin > 96 || a.coutN % 8) return set_error("fv_net: bad convolution shape"), FV_EINVAL;
  switch (a.coutN / 8) {
    case 1: return conv_launch_nt<1>(a, blocks, smem, st);
    case 2: return conv_launch_nt<2>(a, blocks, smem, st);
    case 4: return conv_launch_nt<4>(a, blocks, smem, st);
    case 6: return conv_launch_nt<6>(a, blocks, smem, st);
    case 8: return conv_launch_nt<8>(a, blocks, smem, st);
    case 12: return conv_launch_nt<12>(a, blocks, smem, st);
    default: return set_error("fv_net: unsupported output channel count"), FV_EINVAL;
  }
}

ConvArgs cargs(const bf16* s0, int c0, const bf16* s1, int c1, const bf16* w, int coutN, int cout, int P, int Z,
               int Y, int X, int mode) {
  ConvArgs a{};
  a.s0 = s0, a.c0 = c0, a.s1 = s1, a.c1 = c1, a.cin = c0 + c1, a.w = w, a.coutN = coutN, a.cout = cout;
  a.P = P, a.Z = Z, a.Y = Y, a.X = X, a.mode = mode;
  return a;
}

fv_status wgrad(const fv_net* n, const bf16* s0, int c0, const bf16* s1, int c1, const bf16* g, int gc, int li,
                int P, int Z, int Y, int X, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    FV_CUDA(cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WK * (96 + 8 + 64 + 8) * 2));
    attr = true;
  }
  WGradArgs a{};
  a.s0 = s0, a.c0 = c0, a.s1 = s1, a.c1 = c1, a.cin = c0 + c1, a.g = g, a.gc = gc;
  a.ci = n->L[li].ci, a.co = n->L[li].co, a.gw = n->g + n->L[li].woff;
  a.P = P, a.Z = Z, a.Y = Y, a.X = X;
  if ((a.cin / 16) * (gc / 16) > 4 * WG_PAIRS) return set_error("fv_net: weight-gradient tile too large"), FV_EINVAL;
  const long long V = (long long)P * Z * Y * X, nchunk = (V + WK - 1) / WK;
  const long long groups = std::min<long long>(nchunk, 48);
  a.chunks_per_cta = (nchunk + groups - 1) / groups;
  const dim3 grid((unsigned)((nchunk + a.chunks_per_cta - 1) / a.chunks_per_cta), 27);
  wgrad_kernel<<<grid, CONV_THREADS, (size_t)WK * (a.cin + 8 + gc + 8) * 2, st>>>(a);
  const int rows = RED_THREADS / gc;
  bgrad_kernel<<<gridsz(V, rows) / 4 + 1, RED_THREADS, 0, st>>>(g, gc, a.co, V, n->g + n->L[li].boff);
  return FV_OK;
}

fv_status check_nb(const fv_net* n, int nb) {
  if (!n || nb < 1 || nb > n->nbmax) return set_error("fv_net: batch must be in [1, max_batch]"), FV_EINVAL;
  return FV_OK;
}

// forward pass of nb samples; leaves all activations and y in the network
template <class T>
fv_status forward_t(fv_net* n, int nb, const T* r, cudaStream_t st) {
  const int C = n->C, P = 6 * nb, Z = n->Z, Y = n->Y, X = n->X;
  const long long V = n->V1 * nb;
  FV_CUDA(cudaMemsetAsync(n->ss, 0, nb * sizeof(double), st));
  sumsq_kernel<T><<<dim3(gridsz(2 * n->V1, RED_THREADS) / 8 + 1, nb), RED_THREADS, 0, st>>>(r, 2 * n->V1, n->ss);
  pack_kernel<T><<<gridsz(V, 256), 256, 0, st>>>(r, n->ss, n->V1, nb, n->x);
  fv_status rc;
  ConvArgs a = cargs(n->x, 16, nullptr, 0, n->L[0].wf, C, C, P, Z, Y, X, EPI_RELU);
  a.bias = n->w + n->L[0].boff, a.out = n->a1;
  if ((rc = conv(a, st))) return rc;
  a = cargs(n->a1, C, nullptr, 0, n->L[1].wf, C, C, P, Z, Y, X, EPI_RELU);
  a.bias = n->w + n->L[1].boff, a.out = n->a2;
  if ((rc = conv(a, st))) return rc;
  pool_kernel<<<gridsz(V / 8 * (C / 8), 256), 256, 0, st>>>(n->a2, n->p, C, P, Z, Y, X);
  a = cargs(n->p, C, nullptr, 0, n->L[2].wf, 2 * C, 2 * C, P, Z / 2, Y / 2, X / 2, EPI_RELU);
  a.bias = n->w + n->L[2].boff, a.out = n->a3;
  if ((rc = conv(a, st))) return rc;
  a = cargs(n->a3, 2 * C, nullptr, 0, n->L[3].wf, 2 * C, 2 * C, P, Z / 2, Y / 2, X / 2, EPI_RELU);
  a.bias = n->w + n->L[3].boff, a.out = n->a4;
  if ((rc = conv(a, st))) return rc;
  a = cargs(n->a2, C, n->a4, 2 * C, n->L[4].wf, C, C, P, Z, Y, X, EPI_RELU);
  a.bias = n->w + n->L[4].boff, a.out = n->a5;
  if ((rc = conv(a, st))) return rc;
  a = cargs(n->a5, C, nullptr, 0, n->L[5].wf, 8, 2, P, Z, Y, X, EPI_FINAL);
  a.bias = n->w + n->L[5].boff, a.y = n->y;
  return conv(a, st);
}

fv_status pack_weights(fv_net* n, cudaStream_t st) {
  for (int l = 0; l < 6; ++l) {
    const NetLayer& L = n->L[l];
    const int tot = 27 * L.coN * L.ciK + (L.wb ? 27 * L.ciN * L.coK : 0);
    packw_kernel<<<gridsz(tot, 256), 256, 0, st>>>(n->w + L.woff, L.ci, L.co, L.ciK, L.coN, L.ciN, L.coK, L.wf, L.wb);
  }
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status ensure_train(fv_net* n) {
  if (n->gy) return FV_OK;
  const long long V = n->V1 * n->nbmax, Vh = V / 8;
  const int C = n->C;
  fv_status rc;
  if ((rc = nalloc(n, &n->gy, V * 16)) || (rc = nalloc(n, &n->g5, V * C)) || (rc = nalloc(n, &n->gcat, V * 3 * C)) ||
      (rc = nalloc(n, &n->g4, Vh * 2 * C)) || (rc = nalloc(n, &n->g3, Vh * 2 * C)) || (rc = nalloc(n, &n->gp, Vh * C)) ||
      (rc = nalloc(n, &n->g2, V * C)) || (rc = nalloc(n, &n->g1, V * C)) ||
      (rc = nalloc(n, &n->rb, 2 * n->V1 * n->nbmax)) || (rc = nalloc(n, &n->eb, 2 * n->V1 * n->nbmax)))
    return rc;
  for (int l = 1; l < 6; ++l) {
    NetLayer& L = n->L[l];
    if ((rc = nalloc(n, &L.wb, (size_t)27 * L.ciN * L.coK))) return rc;
  }
  if ((rc = pack_weights(n, 0))) return rc;
  FV_CUDA(cudaDeviceSynchronize());
  return FV_OK;
}


// loss (device n->loss, sum of squares) and the full parameter gradient into n->g
fv_status loss_grad_dev(fv_net* n, int nb, const double* r, const double* e, cudaStream_t st) {
  fv_status rc;
  if ((rc = forward_t<double>(n, nb, r, st))) return rc;
  const int C = n->C, P = 6 * nb, Z = n->Z, Y = n->Y, X = n->X, Zh = Z / 2, Yh = Y / 2, Xh = X / 2;
  const long long V = n->V1 * nb, Vh = V / 8;
  FV_CUDA(cudaMemsetAsync(n->loss, 0, sizeof(double), st));
  FV_CUDA(cudaMemsetAsync(n->g, 0, n->nparam * sizeof(float), st));
  loss_kernel<<<gridsz(V, RED_THREADS) / 4 + 1, RED_THREADS, 0, st>>>(n->y, e, n->ss, n->V1, nb,
                                                                       1.0 / (2.0 * (double)V), n->gy, n->loss);
  // c6: gy -> g5 (mask a5), weight grad from a5
  ConvArgs a = cargs(n->gy, 16, nullptr, 0, n->L[5].wb, C, C, P, Z, Y, X, EPI_MASK);
  a.mask = n->a5, a.out = n->g5;
  if ((rc = conv(a, st)) || (rc = wgrad(n, n->a5, C, nullptr, 0, n->gy, 16, 5, P, Z, Y, X, st))) return rc;
  // c5: g5 -> gcat (raw), weight grad from [a2, up(a4)]
  a = cargs(n->g5, C, nullptr, 0, n->L[4].wb, 3 * C, 3 * C, P, Z, Y, X, EPI_RAW);
  a.out = n->gcat;
  if ((rc = conv(a, st)) || (rc = wgrad(n, n->a2, C, n->a4, 2 * C, n->g5, C, 4, P, Z, Y, X, st))) return rc;
  g4_kernel<<<gridsz(Vh * 2 * C, 256), 256, 0, st>>>(n->gcat, n->a4, n->g4, C, P, Z, Y, X);
  // c4: g4 -> g3 (mask a3)
  a = cargs(n->g4, 2 * C, nullptr, 0, n->L[3].wb, 2 * C, 2 * C, P, Zh, Yh, Xh, EPI_MASK);
  a.mask = n->a3, a.out = n->g3;
  if ((rc = conv(a, st)) || (rc = wgrad(n, n->a3, 2 * C, nullptr, 0, n->g4, 2 * C, 3, P, Zh, Yh, Xh, st))) return rc;
  // c3: g3 -> gp (raw)
  a = cargs(n->g3, 2 * C, nullptr, 0, n->L[2].wb, C, C, P, Zh, Yh, Xh, EPI_RAW);
  a.out = n->gp;
  if ((rc = conv(a, st)) || (rc = wgrad(n, n->p, C, nullptr, 0, n->g3, 2 * C, 2, P, Zh, Yh, Xh, st))) return rc;
  g2_kernel<<<gridsz(V * C, 256), 256, 0, st>>>(n->gcat, n->gp, n->a2, n->g2, C, P, Z, Y, X);
  // c2: g2 -> g1 (mask a1)
  a = cargs(n->g2, C, nullptr, 0, n->L[1].wb, C, C, P, Z, Y, X, EPI_MASK);
  a.mask = n->a1, a.out = n->g1;
  if ((rc = conv(a, st)) || (rc = wgrad(n, n->a1, C, nullptr, 0, n->g2, C, 1, P, Z, Y, X, st))) return rc;
  // c1: weight grad only
  if ((rc = wgrad(n, n->x, 16, nullptr, 0, n->g1, C, 0, P, Z, Y, X, st))) return rc;
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status adam_dev(fv_net* n, const fv_adam_opts* o, cudaStream_t st) {
  if (!o || !(o->lr > 0) || !(o->beta1 >= 0 && o->beta1 < 1) || !(o->beta2 >= 0 && o->beta2 < 1) || !(o->eps > 0))
    return set_error("fv_net: bad Adam options"), FV_EINVAL;
  n->t += 1;
  const double c1 = 1.0 - std::pow(o->beta1, (double)n->t), c2 = 1.0 - std::pow(o->beta2, (double)n->t);
  adam_kernel<<<gridsz(n->nparam, 256), 256, 0, st>>>(n->w, n->g, n->m, n->v, n->nparam, (float)o->lr,
                                                      (float)o->beta1, (float)o->beta2, (float)o->eps, (float)c1,
                                                      (float)c2);
  return pack_weights(n, st);
}

}  // namespace

// ---------------------------------------------------------------- internal entry points (precond.cu)
fv_status net_forward64(fv_net* n, const double* r, double* e, cudaStream_t st) {
  ProfScope ps(FV_K_NET_FWD, st);
  fv_status rc = forward_t<double>(n, 1, r, st);
  if (rc) return rc;
  unpack_kernel<double><<<gridsz(n->V1, 256), 256, 0, st>>>(n->y, n->ss, n->V1, 1, e);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status net_forward32(fv_net* n, const float* r, float* e, cudaStream_t st) {
  ProfScope ps(FV_K_NET_FWD, st);
  fv_status rc = forward_t<float>(n, 1, r, st);
  if (rc) return rc;
  unpack_kernel<float><<<gridsz(n->V1, 256), 256, 0, st>>>(n->y, n->ss, n->V1, 1, e);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

bool net_matches(const fv_net* n, const fv_grid* coarse) {
  return n && coarse && n->Ns == coarse->h.Ns && n->Nr == coarse->h.Nr;
}

}  // namespace fv

using namespace fv;

extern "C" {

fv_status fv_net_create(const fv_net_desc* d, fv_net** out) {
  if (!d || !out) return set_error("fv_net_create: null argument"), FV_EINVAL;
  if ((d->C != 16 && d->C != 32) || d->Ns < 2 || d->Nr < 2 || d->Ns % 2 || d->Nr % 2 || d->max_batch < 1)
    return set_error("fv_net_create: need C in {16, 32}, even Ns, Nr >= 2 and max_batch >= 1"), FV_EINVAL;
  fv_net* n = new fv_net();
  n->C = d->C, n->Ns = d->Ns, n->Nr = d->Nr, n->nbmax = d->max_batch;
  n->Z = d->Nr, n->Y = d->Ns, n->X = d->Ns;
  n->V1 = 6LL * d->Ns * d->Ns * d->Nr;
  const int C = d->C;
  const int io[6][2] = {{2, C}, {C, C}, {C, 2 * C}, {2 * C, 2 * C}, {3 * C, C}, {C, 2}};
  long long off = 0;
  for (int l = 0; l < 6; ++l) {
    NetLayer& L = n->L[l];
    L.ci = io[l][0], L.co = io[l][1];
    L.ciK = r16(L.ci), L.coN = r8(L.co), L.ciN = r8(L.ci), L.coK = r16(L.co);
    L.woff = off, off += 27LL * L.ci * L.co;
    L.boff = off, off += L.co;
  }
  n->nparam = off;
  const long long V = n->V1 * n->nbmax, Vh = V / 8;
  fv_status rc;
  if ((rc = nalloc(n, &n->w, off)) || (rc = nalloc(n, &n->g, off)) || (rc = nalloc(n, &n->m, off)) ||
      (rc = nalloc(n, &n->v, off)) || (rc = nalloc(n, &n->ss, n->nbmax)) || (rc = nalloc(n, &n->loss, 1)) ||
      (rc = nalloc(n, &n->x, V * 16)) || (rc = nalloc(n, &n->a1, V * C)) || (rc = nalloc(n, &n->a2, V * C)) ||
      (rc = nalloc(n, &n->p, Vh * C)) || (rc = nalloc(n, &n->a3, Vh * 2 * C)) || (rc = nalloc(n, &n->a4, Vh * 2 * C)) ||
      (rc = nalloc(n, &n->a5, V * C)) || (rc = nalloc(n, &n->y, V * 2))) {
    fv_net_free(n);
    return rc;
  }
  for (int l = 0; l < 6; ++l)
    if ((rc = nalloc(n, &n->L[l].wf, (size_t)27 * n->L[l].coN * n->L[l].ciK))) {
      fv_net_free(n);
      return rc;
    }
  if (cudaMemset(n->w, 0, off * sizeof(float)) != cudaSuccess || cudaMemset(n->m, 0, off * sizeof(float)) != cudaSuccess ||
      cudaMemset(n->v, 0, off * sizeof(float)) != cudaSuccess || pack_weights(n, 0) != FV_OK ||
      cudaDeviceSynchronize() != cudaSuccess) {
    fv_net_free(n);
    return set_error("fv_net_create: initialisation failed"), FV_ECUDA;
  }
  *out = n;
  return FV_OK;
}

fv_status fv_net_free(fv_net* n) {
  if (!n) return FV_OK;
  for (void* p : n->allocs) cudaFree(p);
  delete n;
  return FV_OK;
}

fv_status fv_net_param_count(const fv_net* n, long long* count) {
  if (!n || !count) return set_error("fv_net_param_count: null argument"), FV_EINVAL;
  *count = n->nparam;
  return FV_OK;
}

fv_status fv_net_set_params(fv_net* n, const float* params) {
  if (!n || !params) return set_error("fv_net_set_params: null argument"), FV_EINVAL;
  FV_CUDA(cudaMemcpy(n->w, params, n->nparam * sizeof(float), cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemset(n->m, 0, n->nparam * sizeof(float)));
  FV_CUDA(cudaMemset(n->v, 0, n->nparam * sizeof(float)));
  n->t = 0;
  fv_status rc = pack_weights(n, 0);
  if (rc) return rc;
  FV_CUDA(cudaDeviceSynchronize());
  return FV_OK;
}

fv_status fv_net_get_params(const fv_net* n, float* params) {
  if (!n || !params) return set_error("fv_net_get_params: null argument"), FV_EINVAL;
  FV_CUDA(cudaDeviceSynchronize());
  FV_CUDA(cudaMemcpy(params, n->w, n->nparam * sizeof(float), cudaMemcpyDeviceToHost));
  return FV_OK;
}

fv_status fv_net_forward(fv_net* n, int nb, const double* r, double* e, void* stream) {
  fv_status rc = check_nb(n, nb);
  if (rc) return rc;
  if (!r || !e || r == e) return set_error("fv_net_forward: bad vectors"), FV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  ProfScope ps(FV_K_NET_FWD, st);
  if ((rc = forward_t<double>(n, nb, r, st))) return rc;
  unpack_kernel<double><<<gridsz(n->V1 * nb, 256), 256, 0, st>>>(n->y, n->ss, n->V1, nb, e);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status fv_net_loss_grad(fv_net* n, int nb, const double* r, const double* e, double* loss, float* grads,
                           void* stream) {
  fv_status rc = check_nb(n, nb);
  if (rc) return rc;
  if (!r || !e) return set_error("fv_net_loss_grad: null vectors"), FV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = ensure_train(n))) return rc;
  {
    ProfScope ps(FV_K_NET_TRAIN, st);
    if ((rc = loss_grad_dev(n, nb, r, e, st))) return rc;
  }
  FV_CUDA(cudaStreamSynchronize(st));
  if (loss) {
    double l;
    FV_CUDA(cudaMemcpy(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost));
    *loss = l / (2.0 * (double)(n->V1 * nb));
  }
  if (grads) FV_CUDA(cudaMemcpy(grads, n->g, n->nparam * sizeof(float), cudaMemcpyDeviceToHost));
  return FV_OK;
}

fv_status fv_net_adam_step(fv_net* n, const float* grads, const fv_adam_opts* opts) {
  if (!n || !grads || !opts) return set_error("fv_net_adam_step: null argument"), FV_EINVAL;
  fv_status rc = ensure_train(n);
  if (rc) return rc;
  FV_CUDA(cudaMemcpy(n->g, grads, n->nparam * sizeof(float), cudaMemcpyHostToDevice));
  if ((rc = adam_dev(n, opts, 0))) return rc;
  FV_CUDA(cudaDeviceSynchronize());
  return FV_OK;
}

fv_status fv_net_train(fv_net* n, int npairs, const double* R, const double* E, const fv_train_opts* o,
                       double* epoch_loss, void* stream) {
  if (!n || !R || !E || !o || npairs < 1 || o->epochs < 0) return set_error("fv_net_train: bad argument"), FV_EINVAL;
  fv_status rc = check_nb(n, o->batch);
  if (rc) return rc;
  if ((rc = ensure_train(n))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ss = (size_t)2 * n->V1;
  std::vector<int> perm(npairs);
  for (int i = 0; i < npairs; ++i) perm[i] = i;
  unsigned long long state = o->seed;
  auto next = [&state]() {  // splitmix64 (Steele, Lea, Flood 2014)
    unsigned long long z = (state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  for (int ep = 0; ep < o->epochs; ++ep) {
    for (int i = npairs - 1; i > 0; --i) std::swap(perm[i], perm[next() % (unsigned long long)(i + 1)]);
    double sum = 0.0;
    int batches = 0;
    for (int b0 = 0; b0 < npairs; b0 += o->batch) {
      const int nb = std::min(o->batch, npairs - b0);
      for (int k = 0; k < nb; ++k) {
        FV_CUDA(cudaMemcpyAsync(n->rb + k * ss, R + (size_t)perm[b0 + k] * ss, ss * sizeof(double),
                                cudaMemcpyDeviceToDevice, st));
        FV_CUDA(cudaMemcpyAsync(n->eb + k * ss, E + (size_t)perm[b0 + k] * ss, ss * sizeof(double),
                                cudaMemcpyDeviceToDevice, st));
      }
      {
        ProfScope ps(FV_K_NET_TRAIN, st);
        if ((rc = loss_grad_dev(n, nb, n->rb, n->eb, st)) || (rc = adam_dev(n, &o->adam, st))) return rc;
      }
      if (epoch_loss) {
        double l;
        FV_CUDA(cudaMemcpyAsync(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        FV_CUDA(cudaStreamSynchronize(st));
        sum += l / (2.0 * (double)(n->V1 * nb));
      }
      ++batches;
    }
    if (epoch_loss) epoch_loss[ep] = sum / batches;
  }
  FV_CUDA(cudaStreamSynchronize(st));
  return FV_OK;
}

}  // extern "C"
