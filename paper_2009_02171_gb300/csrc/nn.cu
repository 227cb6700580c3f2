// Learned coarse correction: a cubed-sphere U-Net on the coarse grid of the
// two-level preconditioner (declared in include/fv_net.h; not in the paper, it
// stands in for the coarse solve of eqn:coarsesolve).
//
// Data layout: activations and gradients are BF16, channels last, one voxel per
// cell of a pyramid level, each panel padded by a one-cell ring in (eta, xi):
// [panel][k][j + 1][i + 1][channel], (Ns_l + 2)^2 voxels a plane, panel = sample
// * 6 + cubed-sphere panel.  The ring holds the neighbouring panel's cells across
// each edge (written by whichever kernel produces the tensor: the convolution epilogue,
// the input packing, the pooling); ring corners stay zero.  A convolution is an implicit
// GEMM (M = voxels, N = output channels, K = 27 taps x input channels) on the
// tensor cores (mma.sync m16n8k16, BF16 x BF16 -> FP32): one CTA computes a
// 4 x 4 x 8 brick of output voxels from a (6 x 6 x 10)-voxel halo of its input
// and all 27 taps' weights, both staged in shared memory (row stride padded by 8
// channels so ldmatrix rows fall in distinct banks).  The backward data pass is the same kernel with flipped,
// transposed weights over the whole padded plane (the gradient of the ring
// included), followed by halo_adjoint (ring gradients added to the neighbour
// cells they were copied from); the weight gradient is a GEMM over voxels
// (M = input channels, N = output channels) split over (tap, voxel range) CTAs,
// whose partial tiles are added in a fixed order (no atomics: training is bitwise
// reproducible).
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
constexpr int MAX_CIN = 64;            // widest convolution input (2C, C <= 32)
constexpr int WK = 64;                 // voxels per weight-gradient chunk
constexpr int RED_THREADS = 256;

enum { EPI_RELU = 0, EPI_RAW = 1, EPI_FINAL = 2 };

// one pyramid level: Z x Y x X cells a panel, stored with the (Y + 2) x (X + 2) ring plane
struct Lvl {
  int Z, Y, X;
  __host__ __device__ long long vox(int P) const { return (long long)P * Z * (Y + 2) * (X + 2); }
  __host__ __device__ long long cells(int P) const { return (long long)P * Z * Y * X; }
};

// Cubed-sphere ring: the ring voxel beyond `side` of panel p at tangential index t takes
// the value of panel q[p][side]'s cell next to its side s[p][side] at tangential index
// t (flip: n - 1 - t).  Sides: 0 xi-min, 1 xi-max, 2 eta-min, 3 eta-max.
struct Halo {
  int q[24], s[24], flip[24];
};

// (y, x) of the cell next to `side` at tangential index t (padded coordinates); ring = outside
__device__ __forceinline__ void side_cell(int side, int t, int n, bool ring, int& y, int& x) {
  const int lo = ring ? 0 : 1, hi = ring ? n + 1 : n;
  if (side == 0) y = t + 1, x = lo;
  else if (side == 1) y = t + 1, x = hi;
  else if (side == 2) y = lo, x = t + 1;
  else y = hi, x = t + 1;
}

// The ring voxels that copy interior cell (pp, z, jj, ii) of a level with n x n cells a plane: one beyond
// each panel edge the cell touches, in the neighbouring panel's ring (the copy a ring voxel takes from the neighbouring panel);
// f(voxel index) stores the value there
template <class F>
__device__ __forceinline__ void ring_targets(const Halo& H, int n, int Z, int pp, int z, int jj, int ii, F&& f) {
  const int pl = pp % 6, base = pp - pl, Yp = n + 2, Xp = n + 2;
#pragma unroll
  for (int sd = 0; sd < 4; ++sd) {
    const bool on = sd == 0 ? ii == 0 : sd == 1 ? ii == n - 1 : sd == 2 ? jj == 0 : jj == n - 1;
    if (!on) continue;
    const int e = pl * 4 + sd, t = sd < 2 ? jj : ii;
    int yr, xr;
    side_cell(H.s[e], H.flip[e] ? n - 1 - t : t, n, true, yr, xr);
    f((((long long)(base + H.q[e]) * Z + z) * Yp + yr) * Xp + xr);
  }
}

struct ConvArgs {
  const bf16* s0;     // input at the output's level, c0 channels (padded)
  const bf16* s1;     // input one level coarser read through nearest upsampling, c1 channels (or null)
  const bf16* w;      // [27][coutN][cin], tap = dz * 9 + dy * 3 + dx, input voxel = output + (dz, dy, dx) - 1
  const float* bias;  // [cout] (RELU, FINAL)
  bf16* out;          // [padded voxel][cout]
  float* y;           // [cell][cout] FP32 (FINAL)
  int c0, c1, cin, coutN, cout;
  int P;
  Lvl L;
  int o0, On;         // output region per plane axis in padded coordinates: [o0, o0 + On) (1, Y: interior; 0, Y + 2: all)
  int i0, i1;         // valid input region per plane axis in padded coordinates, zero outside
  int mode;
  int ring;           // RELU: also write panel-edge outputs into the neighbouring panels' rings
  Halo H;
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

// Address of the 16-byte channel group q (8 channels) of the (possibly concatenated) input at
// padded voxel (p, z, y, x) of level L, or null (value zero) outside the valid region [i0, i1)
// and radially.
__device__ __forceinline__ const bf16* src_in(const bf16* s0, int c0, const bf16* s1, int c1, int q, int p, int z,
                                              int y, int x, const Lvl& L, int i0, int i1) {
  if (z < 0 || z >= L.Z || y < i0 || y >= i1 || x < i0 || x >= i1) return nullptr;
  const int Yp = L.Y + 2, Xp = L.X + 2;
  if (q * 8 < c0) return s0 + ((((long long)p * L.Z + z) * Yp + y) * Xp + x) * c0 + q * 8;
  const int Zh = L.Z >> 1, Yh = (L.Y >> 1) + 2, Xh = (L.X >> 1) + 2;
  const int yh = ((y - 1) >> 1) + 1, xh = ((x - 1) >> 1) + 1;
  return s1 + ((((long long)p * Zh + (z >> 1)) * Yh + yh) * Xh + xh) * c1 + (q * 8 - c0);
}

// asynchronous 16-byte global -> shared copy (zero fill when src is null): a thread's copies are
// all in flight together instead of one round trip per loaded value
__device__ __forceinline__ void cp16(void* dst, const void* src, const void* any) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = src ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src ? src : any), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// NT: output channels / 8 (n tiles), CIN: input channels (a.cin); both fixed at compile time, so the
// staging index arithmetic reduces to shifts and the tap and channel loops unroll
template <int NT, int CIN>
__global__ void __launch_bounds__(CONV_THREADS) conv_kernel(ConvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16* hs = reinterpret_cast<bf16*>(smem_raw);
  constexpr int cs = CIN + 8;
  const int nbx = (a.On + BX - 1) / BX, nby = (a.On + BY - 1) / BY, nbz = (a.L.Z + BZ - 1) / BZ;
  int blk = blockIdx.x;
  const int bx = blk % nbx;
  blk /= nbx;
  const int by = blk % nby;
  blk /= nby;
  const int bz = blk % nbz;
  const int p = blk / nbz;
  const int x0 = a.o0 + bx * BX, y0 = a.o0 + by * BY, z0 = bz * BZ;  // padded coordinates of the brick origin

  constexpr int qn = CIN >> 3;
  for (int it = threadIdx.x; it < HV * qn; it += CONV_THREADS) {
    const int hv = it / qn, q = it - hv * qn;
    const int hx = hv % HX, hy = (hv / HX) % HY, hz = hv / (HX * HY);
    cp16(hs + hv * cs + q * 8,
         src_in(a.s0, a.c0, a.s1, a.c1, q, p, z0 - 1 + hz, y0 - 1 + hy, x0 - 1 + hx, a.L, a.i0, a.i1), a.w);
  }
  // all 27 taps' weights, rows (tap, n) of cin values, staged once: the tap loop then reads the B
  // fragments from shared memory instead of waiting on global loads
  bf16* ws = hs + HV * cs;
  for (int it = threadIdx.x; it < 27 * NT * 8 * qn; it += CONV_THREADS) {
    const int row = it / qn, q = it - row * qn;
    cp16(ws + row * cs + q * 8, a.w + (size_t)row * CIN + q * 8, a.w);
  }
  cp_wait_all();
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
  // B rows: lanes 0-7 / 8-15 give n-tile 2j's rows at k halves 0 / 1, lanes 16-31 n-tile 2j + 1's
  const uint32_t wbase = sbase + (uint32_t)(HV * cs * 2);
  const int brow = ((lane >> 4) * 8 + (lane & 7)), bk = ((lane >> 3) & 1) * 8;
#pragma unroll
  for (int tap = 0; tap < 27; ++tap) {
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    const int toff = (dz * HY + dy) * HX + dx;
#pragma unroll
    for (int kc = 0; kc < CIN; kc += 16) {
      uint32_t af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) ldsm4(sbase + (uint32_t)(((hv0[mt] + toff) * cs + kc + kh * 8) * 2), af[mt]);
#pragma unroll
      for (int np = 0; np < (NT + 1) / 2; ++np) {
        uint32_t bf[4];
        const int row = tap * NT * 8 + np * 16 + (NT == 1 ? (lane & 7) : brow);
        ldsm4(wbase + (uint32_t)((row * cs + kc + bk) * 2), bf);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma16816(acc[mt][2 * np], af[mt], bf[0], bf[1]);
          if (2 * np + 1 < NT) mma16816(acc[mt][2 * np + 1], af[mt], bf[2], bf[3]);
        }
      }
    }
  }

  // epilogue: accumulator e of tile (mt, nt): row (lane >> 2) + 8 (e >> 1), column nt*8 + (lane & 3)*2 + (e & 1)
  const int z = z0 + warp;
  const int Yp = a.L.Y + 2, Xp = a.L.X + 2;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = (lane >> 2) + 8 * h;
      const int y = y0 + 2 * mt + (row >> 3), x = x0 + (row & 7);
      if (z >= a.L.Z || y >= a.o0 + a.On || x >= a.o0 + a.On) continue;
      const long long v = (((long long)p * a.L.Z + z) * Yp + y) * Xp + x;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int col = nt * 8 + (lane & 3) * 2;
        float u0 = acc[mt][nt][2 * h], u1 = acc[mt][nt][2 * h + 1];
        if (a.mode == EPI_FINAL) {  // interior cell index (y, x >= 1 here)
          const long long c = (((long long)p * a.L.Z + z) * a.L.Y + (y - 1)) * a.L.X + (x - 1);
          if (col < a.cout) a.y[c * a.cout + col] = u0 + a.bias[col];
          if (col + 1 < a.cout) a.y[c * a.cout + col + 1] = u1 + a.bias[col + 1];
          continue;
        }
        if (col >= a.cout) continue;
        if (a.mode == EPI_RELU) {
          u0 = fmaxf(u0 + a.bias[col], 0.f);
          u1 = fmaxf(u1 + a.bias[col + 1], 0.f);
        }
        const __nv_bfloat162 o = __floats2bfloat162_rn(u0, u1);
        *reinterpret_cast<__nv_bfloat162*>(a.out + v * a.cout + col) = o;
        if (a.ring)  // the cell is the source of the ring voxel across each panel edge it touches
          ring_targets(a.H, a.L.Y, a.L.Z, p, z, y - 1, x - 1, [&](long long rv) {
            *reinterpret_cast<__nv_bfloat162*>(a.out + rv * a.cout + col) = o;
          });
      }
    }
}

// Adjoint of the ring fill on a gradient over the whole padded plane: every edge cell gets
// the ring gradients copied from it added (1 side, 2 at a panel corner, 4 when n = 1).
// Ring values are left in place (consumers read interior cells only).
__global__ void halo_adjoint_kernel(bf16* __restrict__ g, int C, int P, Lvl L, Halo H) {
  const int n = L.Y;
  const int ne = n > 1 ? 4 * n - 4 : 1;  // edge cells of a plane
  const long long total = (long long)P * L.Z * ne * C;
  const int Yp = L.Y + 2, Xp = L.X + 2;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % C);
    long long t = it / C;
    const int ec = (int)(t % ne);
    t /= ne;
    const int z = (int)(t % L.Z);
    const int pp = (int)(t / L.Z), p = pp % 6, base = pp - p;
    // edge cell ec -> (j, i): bottom row, top row, then the left and right columns without corners
    int j, i;
    if (n == 1) j = 0, i = 0;
    else if (ec < n) j = 0, i = ec;
    else if (ec < 2 * n) j = n - 1, i = ec - n;
    else if (ec < 3 * n - 2) j = ec - 2 * n + 1, i = 0;
    else j = ec - (3 * n - 2) + 1, i = n - 1;
    const long long dst = ((((long long)pp * L.Z + z) * Yp + j + 1) * Xp + i + 1) * C + c;
    float acc = __bfloat162float(g[dst]);
    for (int sq = 0; sq < 4; ++sq) {
      const bool on = sq == 0 ? i == 0 : sq == 1 ? i == n - 1 : sq == 2 ? j == 0 : j == n - 1;
      if (!on) continue;
      const int e = p * 4 + sq;                    // the neighbour across side sq of this panel
      const int tq = sq < 2 ? j : i;               // tangential index on this side
      const int tp = H.flip[e] ? n - 1 - tq : tq;  // ... on the neighbour's side
      int yr, xr;
      side_cell(H.s[e], tp, n, true, yr, xr);
      acc += __bfloat162float(g[((((long long)(base + H.q[e]) * L.Z + z) * Yp + yr) * Xp + xr) * C + c]);
    }
    g[dst] = __float2bfloat16_rn(acc);
  }
}

// g <- g * (a > 0) on interior cells, 0 on the ring (padded tensors of C channels)
__global__ void mask_kernel(bf16* __restrict__ g, const bf16* __restrict__ a, int C, int P, Lvl L) {
  const long long total = L.vox(P) * C;
  const int Yp = L.Y + 2, Xp = L.X + 2;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
    const long long v = it / C;
    const int x = (int)(v % Xp), y = (int)((v / Xp) % Yp);
    const bool in = x >= 1 && x <= L.X && y >= 1 && y <= L.Y;
    g[it] = (in && __bfloat162float(a[it]) > 0.f) ? g[it] : __float2bfloat16_rn(0.f);
  }
}

// interior cell index -> padded voxel index
__device__ __forceinline__ long long padded(long long cell, const Lvl& L) {
  if (cell < 0x7fffffffLL) {  // 32-bit divisions whenever the index fits
    const int c = (int)cell, x = c % L.X, t = c / L.X, y = t % L.Y;
    return ((long long)(t / L.Y) * (L.Y + 2) + y + 1) * (L.X + 2) + x + 1;
  }
  const int x = (int)(cell % L.X);
  long long t = cell / L.X;
  const int y = (int)(t % L.Y);
  t /= L.Y;  // p * Z + z
  return (t * (L.Y + 2) + y + 1) * (L.X + 2) + x + 1;
}

// 2x2x2 mean pooling of the interior of a (level l) into the interior of out (level l + 1 = Lc), and of
// the pooled panel-edge cells into the neighbouring panels' rings
__global__ void pool_kernel(const bf16* __restrict__ a, bf16* __restrict__ out, int C, int P, Lvl Lc, Halo H) {
  const Lvl L{Lc.Z * 2, Lc.Y * 2, Lc.X * 2};
  const int qn = C / 8;
  const long long total = Lc.cells(P) * qn;
  const bool small = total < 0x7fffffffLL;  // 32-bit divisions whenever the index fits
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
    int q, x, y, z;
    long long cell, p;
    if (small) {
      const int i32 = (int)it, c32 = i32 / qn, pz = c32 / (Lc.X * Lc.Y);
      q = i32 - c32 * qn, x = c32 % Lc.X, y = (c32 / Lc.X) % Lc.Y, z = pz % Lc.Z;
      cell = c32, p = pz / Lc.Z;
    } else {
      q = (int)(it % qn);
      cell = it / qn;
      x = (int)(cell % Lc.X), y = (int)((cell / Lc.X) % Lc.Y);
      const long long pz = cell / ((long long)Lc.X * Lc.Y);  // p * Zc + z
      z = (int)(pz % Lc.Z);
      p = pz / Lc.Z;
    }
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = 0; c < 8; ++c) {
      const long long v = (((p * L.Z + 2 * z + (c >> 2)) * (L.Y + 2) + 2 * y + ((c >> 1) & 1) + 1) * (L.X + 2) + 2 * x +
                           (c & 1) + 1);
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
    *reinterpret_cast<uint4*>(out + padded(cell, Lc) * C + q * 8) = o;
    ring_targets(H, Lc.Y, Lc.Z, (int)p, z, y, x, [&](long long rv) { *reinterpret_cast<uint4*>(out + rv * C + q * 8) = o; });
  }
}

// decoder backward split of gcat (2C channels, level l, interior after halo_adjoint):
// gE[child][c] = gcat[child][c] (skip), gnext[parent][c] = sum over children of
// gcat[child][C + c], times (mask[parent][c] > 0) when a mask is given
__global__ void split_kernel(const bf16* __restrict__ gcat, bf16* __restrict__ gE, bf16* __restrict__ gnext,
                             const bf16* __restrict__ mask, int C, int P, Lvl Lc) {
  const Lvl L{Lc.Z * 2, Lc.Y * 2, Lc.X * 2};
  const long long total = Lc.cells(P) * C;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % C);
    const long long cell = it / C;
    const int x = (int)(cell % Lc.X), y = (int)((cell / Lc.X) % Lc.Y);
    const long long pz = cell / ((long long)Lc.X * Lc.Y);
    const int z = (int)(pz % Lc.Z);
    const long long p = pz / Lc.Z;
    float s = 0.f;
    for (int k = 0; k < 8; ++k) {
      const long long v = (((p * L.Z + 2 * z + (k >> 2)) * (L.Y + 2) + 2 * y + ((k >> 1) & 1) + 1) * (L.X + 2) + 2 * x +
                           (k & 1) + 1);
      gE[v * C + c] = gcat[v * 2 * C + c];
      s += __bfloat162float(gcat[v * 2 * C + C + c]);
    }
    const long long pv = padded(cell, Lc) * C + c;
    if (mask && !(__bfloat162float(mask[pv]) > 0.f)) s = 0.f;
    gnext[pv] = __float2bfloat16_rn(s);
  }
}

// encoder backward through the pooling: gE[child] += g[parent] / 8 (interiors; Lc = parent level)
__global__ void unpool_add_kernel(const bf16* __restrict__ g, bf16* __restrict__ gE, int C, int P, Lvl Lc) {
  const Lvl L{Lc.Z * 2, Lc.Y * 2, Lc.X * 2};
  const long long total = L.cells(P) * C;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it % C);
    const long long cell = it / C;
    const int x = (int)(cell % L.X), y = (int)((cell / L.X) % L.Y);
    const long long pz = cell / ((long long)L.X * L.Y);
    const int z = (int)(pz % L.Z);
    const long long p = pz / L.Z;
    const long long pc = ((p * Lc.Z + z / 2) * Lc.Y + y / 2) * Lc.X + x / 2;
    const long long v = padded(cell, L) * C + c;
    gE[v] = __float2bfloat16_rn(__bfloat162float(gE[v]) + 0.125f * __bfloat162float(g[padded(pc, Lc) * C + c]));
  }
}

// Weight gradient of one convolution: gw[co][ci][tap] = sum over interior output cells v of
// in[v + tap offset][ci] * g[v][co].  CTA (chunk group, tap); warp pairs (16 input channels) x
// (16 output channels) accumulate over WK-cell chunks; each CTA stores its partial tile and
// wsum_kernel adds the groups' tiles in a fixed order (bitwise reproducible training).
struct WGradArgs {
  const bf16* s0;
  const bf16* s1;
  const bf16* g;
  float* part;  // [CTA group][tap][co][ci] partial sums (summed in a fixed order: deterministic)
  int c0, c1, cin, gc, ci, co;
  int P;
  Lvl L;
  long long chunks_per_cta;
};

constexpr int WG_PAIRS = 4;     // (16 x 16) output tiles per warp: cin/16 * gc/16 <= 16
constexpr int WG_GROUPS = 48;   // voxel-range groups of the weight gradient (partial tiles)
constexpr int BG_BLOCKS = 640;  // blocks of the bias gradient (partial sums)
constexpr int SS_BLOCKS = 320;  // blocks per sample of the sum of squares

__global__ void __launch_bounds__(CONV_THREADS) wgrad_kernel(WGradArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int xsn = a.cin + 8, gsn = a.gc + 8;
  bf16* xs = reinterpret_cast<bf16*>(smem_raw);
  bf16* gs = xs + WK * xsn;
  const int tap = blockIdx.y;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const long long V = a.L.cells(a.P);
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
      const bf16* src = nullptr;
      if (v < V) {
        long long t = v;
        const int x = (int)(t % a.L.X);
        t /= a.L.X;
        const int y = (int)(t % a.L.Y);
        t /= a.L.Y;
        const int z = (int)(t % a.L.Z);
        const int p = (int)(t / a.L.Z);
        src = src_in(a.s0, a.c0, a.s1, a.c1, qq, p, z + dz, y + 1 + dy, x + 1 + dx, a.L, 0, a.L.Y + 2);
      }
      cp16(xs + k * xsn + qq * 8, src, a.g);
    }
    for (int it = threadIdx.x; it < WK * qg; it += CONV_THREADS) {
      const int k = it / qg, qq = it - k * qg;
      const long long v = ch * WK + k;
      cp16(gs + k * gsn + qq * 8, v < V ? a.g + padded(v, a.L) * a.gc + qq * 8 : nullptr, a.g);
    }
    cp_wait_all();
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
        if (m < a.ci && n < a.co) a.part[((long long)blockIdx.x * 27 + tap) * a.ci * a.co + n * a.ci + m] = acc[i][h][e];
      }
  }
}

// gw[co][ci][tap] = sum over the groups (in order) of the partial tiles
__global__ void wsum_kernel(const float* __restrict__ part, int groups, int ci, int co, float* __restrict__ gw) {
  const int n = 27 * ci * co;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x) {
    const int tap = it % 27, m = (it / 27) % ci, o = it / (27 * ci);
    float s = 0.f;
    for (int g = 0; g < groups; ++g) s += part[((long long)g * 27 + tap) * ci * co + o * ci + m];
    gw[it] = s;
  }
}

// bias gradient, per block: bpart[block][c] = sum over the block's interior cells of g[v][c]
__global__ void bgrad_kernel(const bf16* __restrict__ g, int gc, int co, int P, Lvl L, float* bpart) {
  __shared__ float part[RED_THREADS];
  const int rows = RED_THREADS / gc;  // gc divides RED_THREADS (16, 32, 64)
  const int c = threadIdx.x % gc, r = threadIdx.x / gc;
  const long long V = L.cells(P);
  float s = 0.f;
  for (long long v = (long long)blockIdx.x * rows + r; v < V; v += (long long)gridDim.x * rows)
    s += __bfloat162float(g[padded(v, L) * gc + c]);
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < gc) {
    float t = 0.f;
    for (int k = 0; k < rows; ++k) t += part[k * gc + threadIdx.x];
    if (threadIdx.x < co) bpart[blockIdx.x * co + threadIdx.x] = t;
  }
}

// gb[c] = sum over blocks (in order) of bpart[block][c]
__global__ void bsum_kernel(const float* __restrict__ bpart, int blocks, int co, float* __restrict__ gb) {
  if (threadIdx.x >= co) return;
  float s = 0.f;
  for (int b = 0; b < blocks; ++b) s += bpart[b * co + threadIdx.x];
  gb[threadIdx.x] = s;
}

// per-sample sum of squares of a coarse vector batch (sample b: 2 * V1 values): block partials
// sspart[b][block], added in order by sssum_kernel (the scale s is bitwise reproducible)
template <class T>
__global__ void sumsq_kernel(const T* __restrict__ r, long long n1, double* sspart) {
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
  if (threadIdx.x == 0) sspart[blockIdx.y * gridDim.x + blockIdx.x] = part[0];
}

// one warp a sample: lane l adds the partials l, l + 32, ... (loads issued together), then the
// warp's fixed butterfly; the order is the same on every call
// with the sum, the sample's two scales: pinv[i] = 1 / s (as the FP32 value the packing multiplies by) and
// psc[i] = s, s = sqrt(sum / (2 V1)) the RMS, so no element recomputes them
__global__ void sssum_kernel(const double* __restrict__ sspart, int blocks, int nb, double* ss, long long V1,
                             double* pinv, double* psc) {
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x >> 5; i < nb; i += blockDim.x >> 5) {
    double s = 0.0;
    for (int b0 = 0; b0 < blocks; b0 += 32 * 4) {
      double q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = b0 + u * 32 + lane;
        q[u] = b < blocks ? sspart[i * blocks + b] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) s += q[u];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      ss[i] = s;
      pinv[i] = s > 0.0 ? (double)(float)sqrt(2.0 * (double)V1 / s) : 0.0;
      psc[i] = sqrt(s / (2.0 * (double)V1));
    }
  }
}

// x interior [cell][0..15] = (r_P, r_Pb) / s, zero channels 2..15 (cells sample-major), with
// s the RMS of the sample (ss = its sum of squares over 2 V1 values): O(1) activations
template <class T>
__global__ void pack_kernel(const T* __restrict__ r, const double* __restrict__ pinv, long long V1, int nb, Lvl L,
                            bf16* __restrict__ x, Halo H) {
  const long long n = V1 * nb;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const long long b = nb == 1 ? 0 : v / V1, vl = v - b * V1;
    const float inv = (float)pinv[b];
    uint4 o[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(o);
    h[0] = __floats2bfloat162_rn((float)r[b * 2 * V1 + vl] * inv, (float)r[b * 2 * V1 + V1 + vl] * inv);
    uint4* dst = reinterpret_cast<uint4*>(x + padded(v, L) * 16);
    dst[0] = o[0];
    dst[1] = o[1];
    // panel-edge cells also fill the neighbouring panels' rings
    const int xi = (int)(v % L.X), yj = (int)((v / L.X) % L.Y);
    const long long pz = v / ((long long)L.X * L.Y);
    ring_targets(H, L.Y, L.Z, (int)(pz / L.Z), (int)(pz % L.Z), yj, xi, [&](long long rv) {
      uint4* d = reinterpret_cast<uint4*>(x + rv * 16);
      d[0] = o[0];
      d[1] = o[1];
    });
  }
}

// e[b][c][vl] = s_b * y[cell][c] (s_b the RMS of sample b)
template <class T>
__global__ void unpack_kernel(const float* __restrict__ y, const double* __restrict__ psc, long long V1, int nb,
                              T* __restrict__ e) {
  const long long n = V1 * nb;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const long long b = nb == 1 ? 0 : v / V1, vl = v - b * V1;
    const double s = psc[b];
    e[b * 2 * V1 + vl] = (T)(s * (double)y[2 * v]);
    e[b * 2 * V1 + V1 + vl] = (T)(s * (double)y[2 * v + 1]);
  }
}

// loss = sum over entries of (y - e/s)^2 (accumulated); gy interior = 2 (y - e/s) / ntot in
// channels 0, 1 of 16 (the ring of gy stays zero)
__global__ void loss_kernel(const float* __restrict__ y, const double* __restrict__ e, const double* __restrict__ ss,
                            long long V1, int nb, Lvl L, double inv_ntot, bf16* __restrict__ gy, double* loss) {
  __shared__ double part[RED_THREADS];
  const long long n = V1 * nb;
  double acc = 0.0;
  for (long long v = blockIdx.x * (long long)RED_THREADS + threadIdx.x; v < n; v += (long long)gridDim.x * RED_THREADS) {
    const long long b = v / V1, vl = v - b * V1;
    const double s2 = ss[b];
    const double inv = s2 > 0.0 ? sqrt(2.0 * (double)V1 / s2) : 0.0;
    const double d0 = (double)y[2 * v] - e[b * 2 * V1 + vl] * inv;
    const double d1 = (double)y[2 * v + 1] - e[b * 2 * V1 + V1 + vl] * inv;
    acc += d0 * d0 + d1 * d1;
    uint4 o[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
    reinterpret_cast<__nv_bfloat162*>(o)[0] =
        __floats2bfloat162_rn((float)(2.0 * d0 * inv_ntot), (float)(2.0 * d1 * inv_ntot));
    uint4* dst = reinterpret_cast<uint4*>(gy + padded(v, L) * 16);
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
  int ci, co;              // logical channels
  int ciK, coN, ciN, coK;  // padded: forward input (x16), forward output tile (x8), backward output, backward input
  long long woff, boff;    // offsets of W and b in the flat parameters
  bf16 *wf = nullptr, *wb = nullptr;
};

constexpr int MAX_LEVELS = 4;

}  // namespace fv

struct fv_net {
  int C = 0, Ns = 0, Nr = 0, nbmax = 0, levels = 0;
  fv::Lvl lv[fv::MAX_LEVELS + 1];
  long long V1 = 0;       // coarse cells of one sample (6 Ns^2 Nr)
  long long nparam = 0;
  int nlayer = 0;
  fv::NetLayer L[3 * fv::MAX_LEVELS + 3];  // e0a e0b ... eLa eLb, d(L-1) .. d0, out
  fv::Halo halo{};
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 masters, gradient, Adam moments
  long long t = 0;        // Adam step counter
  double* ss = nullptr;   // [3][nbmax] per-sample sum of squares, then 1 / RMS and RMS
  double* sspart = nullptr;  // [nbmax][SS_BLOCKS] its block partials
  float *wpart = nullptr, *bpart = nullptr;  // weight- and bias-gradient partials (training)
  double* loss = nullptr; // [1]
  // activations (BF16, channels last, padded planes)
  fv::bf16* x0 = nullptr;
  fv::bf16 *A[fv::MAX_LEVELS + 1] = {}, *E[fv::MAX_LEVELS + 1] = {}, *In[fv::MAX_LEVELS + 1] = {},
           *D[fv::MAX_LEVELS + 1] = {};
  float* y = nullptr;     // [cell][2] of level 0
  // gradients (allocated on the first training call)
  fv::bf16 *gy = nullptr, *T = nullptr, *gE[fv::MAX_LEVELS + 1] = {}, *gD[fv::MAX_LEVELS + 1] = {};
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
  if (cudaMemset(*p, 0, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess)
    return set_error("fv_net: device memset failed"), FV_ECUDA;
  return FV_OK;
}

int eA(int l) { return 2 * l; }
int eB(int l) { return 2 * l + 1; }
int dL(const fv_net* n, int l) { return 2 * (n->levels + 1) + (n->levels - 1 - l); }
int outL(const fv_net* n) { return 2 * (n->levels + 1) + n->levels; }

template <int NT, int CIN>
fv_status conv_launch_nt(const ConvArgs& a, int blocks, size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    FV_CUDA(cudaFuncSetAttribute(conv_kernel<NT, CIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  conv_kernel<NT, CIN><<<blocks, CONV_THREADS, smem, st>>>(a);
  return FV_OK;
}

template <int NT>
fv_status conv_launch_cin(const ConvArgs& a, int blocks, size_t smem, cudaStream_t st) {
  switch (a.cin) {
    case 16: return conv_launch_nt<NT, 16>(a, blocks, smem, st);
    case 32: return conv_launch_nt<NT, 32>(a, blocks, smem, st);
    case 48: return conv_launch_nt<NT, 48>(a, blocks, smem, st);
    case 64: return conv_launch_nt<NT, 64>(a, blocks, smem, st);
    default: return set_error("fv_net: unsupported input channel count"), FV_EINVAL;
  }
}

fv_status conv(const ConvArgs& a, cudaStream_t st) {
  const int blocks = a.P * ((a.L.Z + BZ - 1) / BZ) * ((a.On + BY - 1) / BY) * ((a.On + BX - 1) / BX);
  const size_t smem = (size_t)(HV + 27 * a.coutN) * (a.cin + 8) * 2;  // halo + the staged weights
  if (a.cin % 16 || a.c0 % 8 || a.cin > MAX_CIN || a.coutN % 8 || smem > 200 * 1024)
    return set_error("fv_net: bad convolution shape"), FV_EINVAL;
  switch (a.coutN / 8) {
    case 1: return conv_launch_cin<1>(a, blocks, smem, st);
    case 2: return conv_launch_cin<2>(a, blocks, smem, st);
    case 4: return conv_launch_cin<4>(a, blocks, smem, st);
    case 8: return conv_launch_cin<8>(a, blocks, smem, st);
    default: return set_error("fv_net: unsupported output channel count"), FV_EINVAL;
  }
}

// forward convolution: output interior, input with its ring
ConvArgs fwd_args(const bf16* s0, int c0, const bf16* s1, int c1, const NetLayer& ly, int P, const Lvl& L, int mode) {
  ConvArgs a{};
  a.s0 = s0, a.c0 = c0, a.s1 = s1, a.c1 = c1, a.cin = c0 + c1, a.w = ly.wf, a.coutN = ly.coN, a.cout = ly.co;
  a.P = P, a.L = L, a.o0 = 1, a.On = L.Y, a.i0 = 0, a.i1 = L.Y + 2, a.mode = mode;
  return a;
}

// backward data: gradient with respect to the whole padded input plane from an interior-only g
ConvArgs bwd_args(const bf16* g, const NetLayer& ly, bf16* out, int P, const Lvl& L) {
  ConvArgs a{};
  a.s0 = g, a.c0 = ly.coK, a.s1 = nullptr, a.c1 = 0, a.cin = ly.coK, a.w = ly.wb, a.coutN = ly.ciN, a.cout = ly.ciN;
  a.P = P, a.L = L, a.o0 = 0, a.On = L.Y + 2, a.i0 = 1, a.i1 = L.Y + 1, a.mode = EPI_RAW, a.out = out;
  return a;
}

fv_status wgrad(fv_net* n, const bf16* s0, int c0, const bf16* s1, int c1, const bf16* g, int gc, int li, int P,
                const Lvl& L, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    FV_CUDA(cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WK * (MAX_CIN + 8 + 64 + 8) * 2));
    attr = true;
  }
  WGradArgs a{};
  a.s0 = s0, a.c0 = c0, a.s1 = s1, a.c1 = c1, a.cin = c0 + c1, a.g = g, a.gc = gc;
  a.ci = n->L[li].ci, a.co = n->L[li].co, a.part = n->wpart;
  a.P = P, a.L = L;
  if ((a.cin / 16) * (gc / 16) > 4 * WG_PAIRS) return set_error("fv_net: weight-gradient tile too large"), FV_EINVAL;
  const long long V = L.cells(P), nchunk = (V + WK - 1) / WK;
  const long long groups = std::min<long long>(nchunk, WG_GROUPS);
  a.chunks_per_cta = (nchunk + groups - 1) / groups;
  const int ng = (int)((nchunk + a.chunks_per_cta - 1) / a.chunks_per_cta);
  wgrad_kernel<<<dim3(ng, 27), CONV_THREADS, (size_t)WK * (a.cin + 8 + gc + 8) * 2, st>>>(a);
  wsum_kernel<<<gridsz(27LL * a.ci * a.co, 256), 256, 0, st>>>(n->wpart, ng, a.ci, a.co, n->g + n->L[li].woff);
  const int rows = RED_THREADS / gc, nbk = std::min(gridsz(V, rows) / 4 + 1, BG_BLOCKS);
  bgrad_kernel<<<nbk, RED_THREADS, 0, st>>>(g, gc, a.co, P, L, n->bpart);
  bsum_kernel<<<1, 64, 0, st>>>(n->bpart, nbk, a.co, n->g + n->L[li].boff);
  return FV_OK;
}

void halo_adj(fv_net* n, bf16* g, int C, int P, const Lvl& L, cudaStream_t st) {
  const long long ne = L.Y > 1 ? 4 * L.Y - 4 : 1;
  halo_adjoint_kernel<<<gridsz((long long)P * L.Z * ne * C, 256), 256, 0, st>>>(g, C, P, L, n->halo);
}

void mask(bf16* g, const bf16* a, int C, int P, const Lvl& L, cudaStream_t st) {
  mask_kernel<<<gridsz(L.vox(P) * C, 256), 256, 0, st>>>(g, a, C, P, L);
}

fv_status check_nb(const fv_net* n, int nb) {
  if (!n || nb < 1 || nb > n->nbmax) return set_error("fv_net: batch must be in [1, max_batch]"), FV_EINVAL;
  return FV_OK;
}

// forward pass of nb samples; leaves all activations and y in the network
template <class T>
fv_status forward_t(fv_net* n, int nb, const T* r, cudaStream_t st) {
  const int C = n->C, P = 6 * nb, Lv = n->levels;
  const int sblk = std::min(gridsz(2 * n->V1, RED_THREADS) / 8 + 1, SS_BLOCKS);
  sumsq_kernel<T><<<dim3(sblk, nb), RED_THREADS, 0, st>>>(r, 2 * n->V1, n->sspart);
  sssum_kernel<<<1, 256, 0, st>>>(n->sspart, sblk, nb, n->ss, n->V1, n->ss + n->nbmax, n->ss + 2 * n->nbmax);
  pack_kernel<T><<<gridsz(n->V1 * nb, 256), 256, 0, st>>>(r, n->ss + n->nbmax, n->V1, nb, n->lv[0], n->x0, n->halo);
  fv_status rc;
  for (int l = 0; l <= Lv; ++l) {
    const Lvl& L = n->lv[l];
    const bf16* in = n->x0;
    int cin = 16;
    if (l > 0) {
      pool_kernel<<<gridsz(L.cells(P) * (C / 8), 256), 256, 0, st>>>(n->E[l - 1], n->In[l], C, P, L, n->halo);
      in = n->In[l], cin = C;
    }
    ConvArgs a = fwd_args(in, cin, nullptr, 0, n->L[eA(l)], P, L, EPI_RELU);
    a.bias = n->w + n->L[eA(l)].boff, a.out = n->A[l], a.ring = 1, a.H = n->halo;
    if ((rc = conv(a, st))) return rc;
    a = fwd_args(n->A[l], C, nullptr, 0, n->L[eB(l)], P, L, EPI_RELU);
    a.bias = n->w + n->L[eB(l)].boff, a.out = n->E[l], a.ring = 1, a.H = n->halo;
    if ((rc = conv(a, st))) return rc;
  }
  for (int l = Lv - 1; l >= 0; --l) {
    const bf16* up = l + 1 == Lv ? n->E[Lv] : n->D[l + 1];
    ConvArgs a = fwd_args(n->E[l], C, up, C, n->L[dL(n, l)], P, n->lv[l], EPI_RELU);
    a.bias = n->w + n->L[dL(n, l)].boff, a.out = n->D[l], a.ring = 1, a.H = n->halo;
    if ((rc = conv(a, st))) return rc;
  }
  const bf16* last = Lv > 0 ? n->D[0] : n->E[0];
  ConvArgs a = fwd_args(last, C, nullptr, 0, n->L[outL(n)], P, n->lv[0], EPI_FINAL);
  a.bias = n->w + n->L[outL(n)].boff, a.y = n->y;
  return conv(a, st);
}

fv_status pack_weights(fv_net* n, cudaStream_t st) {
  for (int l = 0; l < n->nlayer; ++l) {
    const NetLayer& L = n->L[l];
    const int tot = 27 * L.coN * L.ciK + (L.wb ? 27 * L.ciN * L.coK : 0);
    packw_kernel<<<gridsz(tot, 256), 256, 0, st>>>(n->w + L.woff, L.ci, L.co, L.ciK, L.coN, L.ciN, L.coK, L.wf, L.wb);
  }
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status ensure_train(fv_net* n) {
  if (n->gy) return FV_OK;
  const int C = n->C, P = 6 * n->nbmax;
  fv_status rc;
  if ((rc = nalloc(n, &n->gy, n->lv[0].vox(P) * 16)) || (rc = nalloc(n, &n->T, n->lv[0].vox(P) * 2 * C)) ||
      (rc = nalloc(n, &n->wpart, (size_t)WG_GROUPS * 27 * MAX_CIN * 64)) ||
      (rc = nalloc(n, &n->bpart, (size_t)BG_BLOCKS * 64)) ||
      (rc = nalloc(n, &n->rb, 2 * n->V1 * n->nbmax)) || (rc = nalloc(n, &n->eb, 2 * n->V1 * n->nbmax)))
    return rc;
  for (int l = 0; l <= n->levels; ++l)
    if ((rc = nalloc(n, &n->gE[l], n->lv[l].vox(P) * C)) || (rc = nalloc(n, &n->gD[l], n->lv[l].vox(P) * C))) return rc;
  for (int l = 0; l < n->nlayer; ++l) {
    NetLayer& L = n->L[l];
    if (l == eA(0)) continue;  // the gradient with respect to the input is not needed
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
  const int C = n->C, P = 6 * nb, Lv = n->levels;
  const Lvl& L0 = n->lv[0];
  FV_CUDA(cudaMemsetAsync(n->loss, 0, sizeof(double), st));
  FV_CUDA(cudaMemsetAsync(n->g, 0, n->nparam * sizeof(float), st));
  loss_kernel<<<gridsz(n->V1 * nb, RED_THREADS) / 4 + 1, RED_THREADS, 0, st>>>(
      n->y, e, n->ss, n->V1, nb, L0, 1.0 / (2.0 * (double)(n->V1 * nb)), n->gy, n->loss);
  // output convolution: gradient of its input, D_0 (or E_0 without levels)
  const bf16* last = Lv > 0 ? n->D[0] : n->E[0];
  if ((rc = conv(bwd_args(n->gy, n->L[outL(n)], n->T, P, L0), st)) ||
      (rc = wgrad(n, last, C, nullptr, 0, n->gy, 16, outL(n), P, L0, st)))
    return rc;
  halo_adj(n, n->T, C, P, L0, st);
  FV_CUDA(cudaMemcpyAsync(Lv > 0 ? n->gD[0] : n->gE[0], n->T, L0.vox(P) * C * sizeof(bf16), cudaMemcpyDeviceToDevice,
                          st));
  if (Lv > 0) mask(n->gD[0], n->D[0], C, P, L0, st);
  // decoder, in reverse order of the forward pass
  for (int l = 0; l < Lv; ++l) {
    const Lvl& L = n->lv[l];
    const bf16* up = l + 1 == Lv ? n->E[Lv] : n->D[l + 1];
    if ((rc = conv(bwd_args(n->gD[l], n->L[dL(n, l)], n->T, P, L), st)) ||
        (rc = wgrad(n, n->E[l], C, up, C, n->gD[l], C, dL(n, l), P, L, st)))
      return rc;
    halo_adj(n, n->T, 2 * C, P, L, st);
    bf16* gnext = l + 1 == Lv ? n->gE[Lv] : n->gD[l + 1];
    const bf16* mk = l + 1 == Lv ? nullptr : n->D[l + 1];
    split_kernel<<<gridsz(n->lv[l + 1].cells(P) * C, 256), 256, 0, st>>>(n->T, n->gE[l], gnext, mk, C, P, n->lv[l + 1]);
  }
  // encoder, from the bottom level up
  for (int l = Lv; l >= 0; --l) {
    const Lvl& L = n->lv[l];
    mask(n->gE[l], n->E[l], C, P, L, st);
    if ((rc = conv(bwd_args(n->gE[l], n->L[eB(l)], n->T, P, L), st)) ||
        (rc = wgrad(n, n->A[l], C, nullptr, 0, n->gE[l], C, eB(l), P, L, st)))
      return rc;
    halo_adj(n, n->T, C, P, L, st);
    bf16* gA = n->gD[l];  // free at this point: holds the gradient of A_l's pre-activation
    FV_CUDA(cudaMemcpyAsync(gA, n->T, L.vox(P) * C * sizeof(bf16), cudaMemcpyDeviceToDevice, st));
    mask(gA, n->A[l], C, P, L, st);
    const bf16* in = l > 0 ? n->In[l] : n->x0;
    const int cin = l > 0 ? C : 16;
    if ((rc = wgrad(n, in, cin, nullptr, 0, gA, C, eA(l), P, L, st))) return rc;
    if (l > 0) {
      if ((rc = conv(bwd_args(gA, n->L[eA(l)], n->T, P, L), st))) return rc;
      halo_adj(n, n->T, C, P, L, st);
      unpool_add_kernel<<<gridsz(n->lv[l - 1].cells(P) * C, 256), 256, 0, st>>>(n->T, n->gE[l - 1], C, P, L);
    }
  }
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
  unpack_kernel<double><<<gridsz(n->V1, 256), 256, 0, st>>>(n->y, n->ss + 2 * n->nbmax, n->V1, 1, e);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

fv_status net_forward32(fv_net* n, const float* r, float* e, cudaStream_t st) {
  ProfScope ps(FV_K_NET_FWD, st);
  fv_status rc = forward_t<float>(n, 1, r, st);
  if (rc) return rc;
  unpack_kernel<float><<<gridsz(n->V1, 256), 256, 0, st>>>(n->y, n->ss + 2 * n->nbmax, n->V1, 1, e);
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
  const int Lv = d->levels;
  const int k = 1 << std::max(0, std::min(Lv, MAX_LEVELS));
  if ((d->C != 16 && d->C != 32) || Lv < 0 || Lv > MAX_LEVELS || d->Ns < 1 || d->Nr < 1 || d->Ns % k || d->Nr % k ||
      d->max_batch < 1)
    return set_error("fv_net_create: need C in {16, 32}, levels in [0, 4], Ns and Nr >= 1 divisible by 2^levels, "
                     "max_batch >= 1"),
           FV_EINVAL;
  // panel adjacency from the grid's own edge tables: neighbour panel, its side, orientation
  fv_grid* g = nullptr;
  const fv_grid_desc gd{4, 2, 0.5, 1.5};
  fv_status rc = build_grid(&gd, &g);
  if (rc) return rc;
  fv_net* n = new fv_net();
  for (int e = 0; e < 24; ++e) {
    n->halo.q[e] = g->h.pq[e], n->halo.s[e] = g->h.psq[e];
    n->halo.flip[e] = g->h.ptmap[e * 4 + 0] != 0;
  }
  free_grid(g);
  n->C = d->C, n->Ns = d->Ns, n->Nr = d->Nr, n->nbmax = d->max_batch, n->levels = Lv;
  for (int l = 0; l <= Lv; ++l) n->lv[l] = Lvl{d->Nr >> l, d->Ns >> l, d->Ns >> l};
  n->V1 = 6LL * d->Ns * d->Ns * d->Nr;
  const int C = d->C;
  n->nlayer = 2 * (Lv + 1) + Lv + 1;
  long long off = 0;
  for (int l = 0; l < n->nlayer; ++l) {
    NetLayer& L = n->L[l];
    if (l < 2 * (Lv + 1)) L.ci = (l == 0 ? 2 : C), L.co = C;
    else if (l < 2 * (Lv + 1) + Lv) L.ci = 2 * C, L.co = C;
    else L.ci = C, L.co = 2;
    L.ciK = r16(L.ci), L.coN = r8(L.co), L.ciN = r8(L.ci), L.coK = r16(L.co);
    L.woff = off, off += 27LL * L.ci * L.co;
    L.boff = off, off += L.co;
  }
  n->nparam = off;
  const int P = 6 * n->nbmax;
  if ((rc = nalloc(n, &n->w, off)) || (rc = nalloc(n, &n->g, off)) || (rc = nalloc(n, &n->m, off)) ||
      (rc = nalloc(n, &n->v, off)) || (rc = nalloc(n, &n->ss, 3 * n->nbmax)) || (rc = nalloc(n, &n->loss, 1)) ||
      (rc = nalloc(n, &n->sspart, (size_t)n->nbmax * SS_BLOCKS)) ||
      (rc = nalloc(n, &n->x0, n->lv[0].vox(P) * 16)) || (rc = nalloc(n, &n->y, n->V1 * n->nbmax * 2))) {
    fv_net_free(n);
    return rc;
  }
  for (int l = 0; l <= Lv && !rc; ++l) {
    const long long vx = n->lv[l].vox(P) * C;
    rc = nalloc(n, &n->A[l], vx);
    if (!rc) rc = nalloc(n, &n->E[l], vx);
    if (!rc && l > 0) rc = nalloc(n, &n->In[l], vx);
    if (!rc && l < Lv) rc = nalloc(n, &n->D[l], vx);
  }
  for (int l = 0; l < n->nlayer && !rc; ++l) rc = nalloc(n, &n->L[l].wf, (size_t)27 * n->L[l].coN * n->L[l].ciK);
  if (rc || pack_weights(n, 0) != FV_OK || cudaDeviceSynchronize() != cudaSuccess) {
    fv_net_free(n);
    return rc ? rc : (set_error("fv_net_create: initialisation failed"), FV_ECUDA);
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

fv_status fv_net_init(fv_net* n, unsigned long long seed) {
  if (!n) return set_error("fv_net_init: null network"), FV_EINVAL;
  // He initialisation: W ~ N(0, 2 / (27 ci)), b = 0.  Normals by Box-Muller from
  // 53-bit uniforms in (0, 1) of the splitmix64 stream started at `seed`.
  std::vector<float> w(n->nparam, 0.f);
  unsigned long long state = seed;
  auto next = [&state]() {
    unsigned long long z = (state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  auto uniform = [&]() { return ((double)(next() >> 11) + 0.5) / 9007199254740992.0; };
  for (int l = 0; l < n->nlayer; ++l) {
    const NetLayer& L = n->L[l];
    const double sd = std::sqrt(2.0 / (27.0 * L.ci));
    const long long cnt = 27LL * L.ci * L.co;
    for (long long i = 0; i < cnt; i += 2) {
      const double r = std::sqrt(-2.0 * std::log(uniform())), t = 2.0 * M_PI * uniform();
      w[L.woff + i] = (float)(sd * r * std::cos(t));
      if (i + 1 < cnt) w[L.woff + i + 1] = (float)(sd * r * std::sin(t));
    }
  }
  return fv_net_set_params(n, w.data());
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
  unpack_kernel<double><<<gridsz(n->V1 * nb, 256), 256, 0, st>>>(n->y, n->ss + 2 * n->nbmax, n->V1, nb, e);
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
