// The registration hot path on 3D periodic grids (d = 3; the paper's
// formulation is written for d = 2 or 3, §2-§3, and names 3D as its next
// step). The same method as the 2D library for a compressible problem with
// the spectral preconditioner: RK2 departure points, periodic tricubic
// interpolation (B-spline prefilter by separable recursions, or cubic
// Lagrange), the semi-Lagrangian state, adjoint, incremental state and
// Gauss-Newton incremental adjoint steps (§3.3.2), pseudospectral grad, div
// and (beta A)^s by 3D FFTs (a complex pass per axis, fft_axis), J, the
// reduced gradient, the GN Hessian matvec and the inexact Newton-Krylov
// solve with P_REG (§3.4).
//
// Layout: a scalar field is n1 n2 n3 float32 with x_1 fastest, then x_2,
// then x_3 (u[(k n2 + j) n1 + i]); a vector field its three components back
// to back. Displacements are stored in cell units.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "common.cuh"
#include "interp.cuh"
#include "kernels.h"
#include "reg.h"

namespace regnk {
namespace d3 {

constexpr int kT = 256;   // threads per block of the pointwise kernels

struct Dims {
  int n1, n2, n3;
  long long N;
};

__device__ __forceinline__ void split3(long long idx, const Dims& d, int& i, int& j, int& k) {
  i = (int)(idx % d.n1);
  const long long r = idx / d.n1;
  j = (int)(r % d.n2);
  k = (int)(r / d.n2);
}

// --------------------------------------------------------------------------
// Tricubic interpolation at node (i, j, k) + (d1, d2, d3) cells: the tensor
// product of the 1D cubic weights over the 4 x 4 x 4 periodic stencil.
struct Stencil3 {
  int ii[4];
  long long jj[4], kk[4];
  float w1[4], w2[4], w3[4];
};

__device__ __forceinline__ Stencil3 stencil3(int i, int j, int k, float d1, float d2, float d3,
                                             const Dims& d, bool lagrange) {
  Stencil3 S;
  const float f1 = floorf(d1), f2 = floorf(d2), f3 = floorf(d3);
  cubic_weights(d1 - f1, S.w1, lagrange);
  cubic_weights(d2 - f2, S.w2, lagrange);
  cubic_weights(d3 - f3, S.w3, lagrange);
  const int i0 = wrap_index<false>(i + (int)f1 - 1, d.n1);
  const int j0 = wrap_index<false>(j + (int)f2 - 1, d.n2);
  const int k0 = wrap_index<false>(k + (int)f3 - 1, d.n3);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int ia = i0 + a, ja = j0 + a, ka = k0 + a;
    S.ii[a] = ia < d.n1 ? ia : ia - d.n1;
    S.jj[a] = (long long)(ja < d.n2 ? ja : ja - d.n2) * d.n1;
    S.kk[a] = (long long)(ka < d.n3 ? ka : ka - d.n3) * d.n1 * d.n2;
  }
  return S;
}

__device__ __forceinline__ float apply3(const Stencil3& S, const float* __restrict__ c) {
  float acc = 0.f;
#pragma unroll
  for (int cz = 0; cz < 4; ++cz) {
    float accy = 0.f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float* row = c + S.kk[cz] + S.jj[b];
      const float r = S.w1[0] * __ldg(row + S.ii[0]) + S.w1[1] * __ldg(row + S.ii[1]) +
                      S.w1[2] * __ldg(row + S.ii[2]) + S.w1[3] * __ldg(row + S.ii[3]);
      accy = fmaf(S.w2[b], r, accy);
    }
    acc = fmaf(S.w3[cz], accy, acc);
  }
  return acc;
}

// Departure points of both characteristics (Heun, §3.3.2), cell units:
// X* = x - a, X_D = x - (a + s v(X*)) / 2 and Y* = x + a, Y_D = x + (a +
// s v(Y*)) / 2 with a = s v, s = h_t n / (2 pi) per axis; cv holds the
// interpolation coefficients of v (or v itself, Lagrange).
__global__ void __launch_bounds__(kT)
k3_departure(Dims d, float s1, float s2, float s3, const float* __restrict__ v,
             const float* __restrict__ cv, float* __restrict__ dX, float* __restrict__ dY,
             int lagrange) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= d.N) return;
  int i, j, k;
  split3(idx, d, i, j, k);
  const long long N = d.N;
  const float a1 = s1 * __ldg(v + idx), a2 = s2 * __ldg(v + N + idx), a3 = s3 * __ldg(v + 2 * N + idx);
  {
    const Stencil3 S = stencil3(i, j, k, -a1, -a2, -a3, d, lagrange);
    dX[idx] = -0.5f * (a1 + s1 * apply3(S, cv));
    dX[N + idx] = -0.5f * (a2 + s2 * apply3(S, cv + N));
    dX[2 * N + idx] = -0.5f * (a3 + s3 * apply3(S, cv + 2 * N));
  }
  {
    const Stencil3 S = stencil3(i, j, k, a1, a2, a3, d, lagrange);
    dY[idx] = 0.5f * (a1 + s1 * apply3(S, cv));
    dY[N + idx] = 0.5f * (a2 + s2 * apply3(S, cv + N));
    dY[2 * N + idx] = 0.5f * (a3 + s3 * apply3(S, cv + 2 * N));
  }
}

// out_f = I[coef_f](x + disp), F fields N apart
__global__ void __launch_bounds__(kT)
k3_gather(Dims d, const float* __restrict__ coef, const float* __restrict__ disp,
          float* __restrict__ out, int F, int lagrange) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= d.N) return;
  int i, j, k;
  split3(idx, d, i, j, k);
  const long long N = d.N;
  const Stencil3 S = stencil3(i, j, k, __ldg(disp + idx), __ldg(disp + N + idx),
                              __ldg(disp + 2 * N + idx), d, lagrange);
  for (int f = 0; f < F; ++f) out[f * N + idx] = apply3(S, coef + f * N);
}

// --------------------------------------------------------------------------
// B-spline prefilter along one axis with whole lines in shared memory: a
// block stages 32 lines (axis 0: 32 consecutive rows; axes 1 and 2: the
// lines through 32 consecutive x_1 of one plane) with coalesced loads; the
// thread (lane, warp) runs the recursions of interp.cuh for the 32-point
// segment `warp` of line `lane` from a chain of kL + 32 + kL samples
// wrapped periodically in shared memory, and the block writes the
// coefficients back with coalesced stores. blockDim.x = n (the line
// length), blockIdx.y the field. Shared layout: axis 0 [line][n + 1] (odd
// pitch), axes 1 and 2 [position][32]: a warp's 32 lines fall in 32 banks.
constexpr int kPSeg = 32;   // outputs per recursion chain

template <int AXIS>
__global__ void __launch_bounds__(256)
k3_prefilter_lines(const float* __restrict__ in, float* __restrict__ out, Dims d) {
  pdl_enter();
  extern __shared__ float sl[];
  const int n = AXIS == 0 ? d.n1 : (AXIS == 1 ? d.n2 : d.n3);
  const int t = threadIdx.x, lane = t & 31, seg = t >> 5;
  in += (long long)blockIdx.y * d.N;
  out += (long long)blockIdx.y * d.N;
  long long base = 0, pstride = 1;
  if (AXIS == 0) {
    base = (long long)blockIdx.x * 32 * d.n1;
  } else {
    const int nx = d.n1 >> 5;
    const long long r = blockIdx.x / nx;
    const int x0 = (int)(blockIdx.x - r * nx) * 32;
    if (AXIS == 1) {
      base = r * d.n2 * d.n1 + x0;
      pstride = d.n1;
    } else {
      base = r * d.n1 + x0;
      pstride = (long long)d.n1 * d.n2;
    }
  }
  const int nw = n >> 5;   // warps = segments per line
  // element e = t + it * n of the block: axis 0 line it, position t; axes 1
  // and 2 position t / 32 + it * nw, line lane
#pragma unroll 8
  for (int it = 0; it < 32; ++it) {
    if (AXIS == 0) {
      sl[it * (n + 1) + t] = __ldg(in + base + (long long)it * n + t);
    } else {
      const int p = seg + it * nw;
      sl[p * 32 + lane] = __ldg(in + base + p * pstride + lane);
    }
  }
  __syncthreads();
  constexpr int NS = kPSeg + 2 * kL;
  float v[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const int p = wrap_once(seg * kPSeg - kL + q, n);
    v[q] = AXIS == 0 ? sl[lane * (n + 1) + p] : sl[p * 32 + lane];
  }
  bspline_recursions<NS, kPSeg>(v, [&](int o, float x) { v[o + kL] = x; });
  __syncthreads();
#pragma unroll
  for (int o = 0; o < kPSeg; ++o) {
    const int p = seg * kPSeg + o;
    if (AXIS == 0) sl[lane * (n + 1) + p] = v[o + kL];
    else sl[p * 32 + lane] = v[o + kL];
  }
  __syncthreads();
#pragma unroll 8
  for (int it = 0; it < 32; ++it) {
    if (AXIS == 0) {
      out[base + (long long)it * n + t] = sl[it * (n + 1) + t];
    } else {
      const int p = seg + it * nw;
      out[base + p * pstride + lane] = sl[p * 32 + lane];
    }
  }
}

// --------------------------------------------------------------------------
// Tricubic gathers from a shared-memory box. A block of 256 threads owns a
// 32 x 8 x 8 tile of points, thread (tx, ty) the eight points (i0 + tx,
// j0 + ty, k0 + tz); the coefficients of the tile widened by h_a cells on
// both sides of axis a are staged in shared memory and every tap of every
// stencil reads them there. With |displacement_a| <= D_a the taps
// floor(d) - 1 .. floor(d) + 2 lie between ceil(D_a) + 1 cells below and
// floor(D_a) + 2 cells above the point, the box's margins; the stencil base
// is clamped to the box all the same, so no access leaves it whatever the
// displacements hold. Box rows are 64 floats apart (a multiple of the 32
// banks), so lanes whose stencils fall on different rows or planes read
// different banks.
constexpr int kBX = 32, kBY = 8, kBZ = 8, kBT = 256;
constexpr int kBMinBlocks = 3;   // resident blocks per SM the register budget allows

constexpr int kBoxPitch = 64;   // floats per box row (b1 <= 64)

struct Box3 {
  int h1, h2, h3;   // lower margin per axis (cells): the box starts h_a before the tile
  int b1, b2, b3;   // box extents: tile + lower + upper margin
};

__device__ __forceinline__ void tile_origin(const Dims& d, int& i0, int& j0, int& k0) {
  const int nx = d.n1 / kBX, ny = d.n2 / kBY;
  const int b = blockIdx.x;
  const int r = b / nx;
  i0 = (b - r * nx) * kBX;
  j0 = (r % ny) * kBY;
  k0 = (r / ny) * kBZ;
}

// stage the box of field c with asynchronous 4-byte copies (every copy of
// the block in flight at once, no registers held): warp w copies the box
// rows (bz, by) with by = w, w + 8, ..., lane the columns lane and lane + 32
// (b1 <= 64); ends with the wait and a block barrier
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src) : "memory");
}

__device__ __forceinline__ void stage_box(const float* __restrict__ c, float* __restrict__ sm,
                                          const Dims& d, const Box3& g, int i0, int j0, int k0) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int xa = wrap_once(i0 - g.h1 + lane, d.n1);
  const bool two = lane + 32 < g.b1;
  const int xb = two ? wrap_once(i0 - g.h1 + lane + 32, d.n1) : 0;
  for (int bz = 0; bz < g.b3; ++bz) {
    const long long zrow = (long long)wrap_once(k0 - g.h3 + bz, d.n3) * d.n2;
    for (int by = w; by < g.b2; by += kBT / 32) {
      const float* row = c + (zrow + wrap_once(j0 - g.h2 + by, d.n2)) * d.n1;
      float* srow = sm + (bz * g.b2 + by) * kBoxPitch;
      cp_async4(srow + lane, row + xa);
      if (two) cp_async4(srow + lane + 32, row + xb);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
}

struct BoxSt {
  int base;   // shared offset of tap (0, 0, 0)
  float w1[4], w2[4], w3[4];
};

__device__ __forceinline__ BoxSt box_stencil(int tx, int ty, int tz, float d1, float d2, float d3,
                                             const Box3& g, bool lagrange) {
  BoxSt S;
  const float f1 = floorf(d1), f2 = floorf(d2), f3 = floorf(d3);
  cubic_weights(d1 - f1, S.w1, lagrange);
  cubic_weights(d2 - f2, S.w2, lagrange);
  cubic_weights(d3 - f3, S.w3, lagrange);
  const int x = min(max(tx + g.h1 + (int)f1 - 1, 0), g.b1 - 4);
  const int y = min(max(ty + g.h2 + (int)f2 - 1, 0), g.b2 - 4);
  const int z = min(max(tz + g.h3 + (int)f3 - 1, 0), g.b3 - 4);
  S.base = (z * g.b2 + y) * kBoxPitch + x;
  return S;
}

__device__ __forceinline__ float box_apply(const BoxSt& S, const float* __restrict__ sm,
                                           const Box3& g) {
  const int plane = kBoxPitch * g.b2;
  float acc = 0.f;
#pragma unroll
  for (int cz = 0; cz < 4; ++cz) {
    float accy = 0.f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float* row = sm + S.base + cz * plane + b * kBoxPitch;
      const float r = S.w1[0] * row[0] + S.w1[1] * row[1] + S.w1[2] * row[2] + S.w1[3] * row[3];
      accy = fmaf(S.w2[b], r, accy);
    }
    acc = fmaf(S.w3[cz], accy, acc);
  }
  return acc;
}

__device__ __forceinline__ long long tile_index(const Dims& d, int i0, int j0, int k0, int tx,
                                                int ty, int tz) {
  return ((long long)(k0 + tz) * d.n2 + (j0 + ty)) * d.n1 + i0 + tx;
}

// The point loops below load the displacement of the next point while the
// current one is evaluated (the first one during the staging), and issue the
// streamed loads of a point before its 64 shared-memory taps.
struct Disp3 {
  float x, y, z;
};

__device__ __forceinline__ Disp3 load_disp(const float* __restrict__ p, long long N, long long idx) {
  return Disp3{__ldg(p + idx), __ldg(p + N + idx), __ldg(p + 2 * N + idx)};
}

// out_f = I[coef_f](x + disp) for F fields N apart (box form of k3_gather)
__global__ void __launch_bounds__(kBT, kBMinBlocks)
k3b_gather(Dims d, Box3 g, const float* __restrict__ coef, const float* __restrict__ disp,
           float* __restrict__ out, int F, int lagrange) {
  pdl_enter();
  extern __shared__ float sbox[];
  int i0, j0, k0;
  tile_origin(d, i0, j0, k0);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long N = d.N, zs = (long long)d.n1 * d.n2;
  const long long idx0 = tile_index(d, i0, j0, k0, tx, ty, 0);
  for (int f = 0; f < F; ++f) {
    Disp3 e = load_disp(disp, N, idx0);
    if (f) __syncthreads();
    stage_box(coef + f * N, sbox, d, g, i0, j0, k0);
#pragma unroll 2
    for (int tz = 0; tz < kBZ; ++tz) {
      const long long idx = idx0 + tz * zs;
      const Disp3 c = e;
      if (tz + 1 < kBZ) e = load_disp(disp, N, idx + zs);
      const BoxSt S = box_stencil(tx, ty, tz, c.x, c.y, c.z, g, lagrange);
      out[f * N + idx] = box_apply(S, sbox, g);
    }
  }
}

// departure points of both characteristics (box form of k3_departure; the
// box of each component of cv covers the reach of s v)
__global__ void __launch_bounds__(kBT, kBMinBlocks)
k3b_departure(Dims d, Box3 g, float s1, float s2, float s3, const float* __restrict__ v,
              const float* __restrict__ cv, float* __restrict__ dX, float* __restrict__ dY,
              int lagrange) {
  pdl_enter();
  extern __shared__ float sbox[];
  int i0, j0, k0;
  tile_origin(d, i0, j0, k0);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long N = d.N, zs = (long long)d.n1 * d.n2;
  const long long idx0 = tile_index(d, i0, j0, k0, tx, ty, 0);
  for (int f = 0; f < 3; ++f) {
    Disp3 e = load_disp(v, N, idx0);
    if (f) __syncthreads();
    stage_box(cv + f * N, sbox, d, g, i0, j0, k0);
    const float sf = f == 0 ? s1 : (f == 1 ? s2 : s3);
#pragma unroll 2
    for (int tz = 0; tz < kBZ; ++tz) {
      const long long idx = idx0 + tz * zs;
      const float a1 = s1 * e.x, a2 = s2 * e.y, a3 = s3 * e.z;
      if (tz + 1 < kBZ) e = load_disp(v, N, idx + zs);
      const float af = f == 0 ? a1 : (f == 1 ? a2 : a3);
      const BoxSt Sm = box_stencil(tx, ty, tz, -a1, -a2, -a3, g, lagrange);
      dX[f * N + idx] = -0.5f * (af + sf * box_apply(Sm, sbox, g));
      const BoxSt Sp = box_stencil(tx, ty, tz, a1, a2, a3, g, lagrange);
      dY[f * N + idx] = 0.5f * (af + sf * box_apply(Sp, sbox, g));
    }
  }
}

// one backward (incremental) adjoint step (box form of k3_adjoint_step)
__global__ void __launch_bounds__(kBT, kBMinBlocks)
k3b_adjoint_step(Dims d, Box3 g, float ht, float wb, const float* __restrict__ coef,
                 const float* __restrict__ dY, const float* __restrict__ delta,
                 const float* __restrict__ delta_bar, const float* __restrict__ gm,
                 float* __restrict__ lam_out, float* __restrict__ b, int lagrange) {
  pdl_enter();
  extern __shared__ float sbox[];
  int i0, j0, k0;
  tile_origin(d, i0, j0, k0);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long N = d.N, zs = (long long)d.n1 * d.n2;
  const long long idx0 = tile_index(d, i0, j0, k0, tx, ty, 0);
  Disp3 e = load_disp(dY, N, idx0);
  stage_box(coef, sbox, d, g, i0, j0, k0);
#pragma unroll 1
  for (int tz = 0; tz < kBZ; ++tz) {
    const long long idx = idx0 + tz * zs;
    const Disp3 c = e;
    if (tz + 1 < kBZ) e = load_disp(dY, N, idx + zs);
    const float db = __ldg(delta_bar + idx), dl = __ldg(delta + idx);
    float gv[3], bv[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      gv[q] = __ldg(gm + q * N + idx);
      bv[q] = b[q * N + idx];
    }
    const BoxSt S = box_stencil(tx, ty, tz, c.x, c.y, c.z, g, lagrange);
    const float lb = box_apply(S, sbox, g);
    const float lstar = fmaf(ht * lb, db, lb);
    const float l = lb + 0.5f * ht * (lb * db + lstar * dl);
    lam_out[idx] = l;
#pragma unroll
    for (int q = 0; q < 3; ++q) b[q * N + idx] = fmaf(wb * l, gv[q], bv[q]);
  }
}

// one forward step of the incremental state (box form of k3_incstate_step):
// the first step gathers the three components of v~ at X_D (stored in vtD)
// and starts from m~_0 = 0, the others gather m~_{j-1}
__global__ void __launch_bounds__(kBT, kBMinBlocks)
k3b_incstate_step(Dims d, Box3 g, float ht, const float* __restrict__ coef,
                  const float* __restrict__ dX, const float* __restrict__ vt,
                  float* __restrict__ vtD, const float* __restrict__ G,
                  const float* __restrict__ gm, float* __restrict__ out, int first,
                  const float* __restrict__ cvt, int lagrange) {
  pdl_enter();
  extern __shared__ float sbox[];
  int i0, j0, k0;
  tile_origin(d, i0, j0, k0);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long N = d.N, zs = (long long)d.n1 * d.n2;
  const long long idx0 = tile_index(d, i0, j0, k0, tx, ty, 0);
  if (first) {
    for (int c = 0; c < 3; ++c) {
      Disp3 e = load_disp(dX, N, idx0);
      if (c) __syncthreads();
      stage_box(cvt + c * N, sbox, d, g, i0, j0, k0);
#pragma unroll 1
      for (int tz = 0; tz < kBZ; ++tz) {
        const long long idx = idx0 + tz * zs;
        const Disp3 q = e;
        if (tz + 1 < kBZ) e = load_disp(dX, N, idx + zs);
        const BoxSt S = box_stencil(tx, ty, tz, q.x, q.y, q.z, g, lagrange);
        vtD[c * N + idx] = box_apply(S, sbox, g);
      }
    }
  }
  Disp3 e{0.f, 0.f, 0.f};
  if (!first) {
    e = load_disp(dX, N, idx0);
    stage_box(coef, sbox, d, g, i0, j0, k0);
  }
#pragma unroll 1
  for (int tz = 0; tz < kBZ; ++tz) {
    const long long idx = idx0 + tz * zs;
    const Disp3 q = e;
    if (!first && tz + 1 < kBZ) e = load_disp(dX, N, idx + zs);
    float w[3], Gv[3], vv[3], gv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      w[c] = vtD[c * N + idx];
      Gv[c] = __ldg(G + c * N + idx);
      vv[c] = __ldg(vt + c * N + idx);
      gv[c] = __ldg(gm + c * N + idx);
    }
    float m = 0.f;
    if (!first) {
      const BoxSt S = box_stencil(tx, ty, tz, q.x, q.y, q.z, g, lagrange);
      m = box_apply(S, sbox, g);
    }
    float src = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) src += w[c] * Gv[c] + vv[c] * gv[c];
    out[idx] = m - 0.5f * ht * src;
  }
}

// lambda = sign (mR - m1) (mR may be NULL), b = coef_b lambda grad m
__global__ void __launch_bounds__(kT)
k3_adjoint_init(long long N, float coef_b, const float* __restrict__ mR,
                const float* __restrict__ m1, const float* __restrict__ gm,
                float* __restrict__ lam, float* __restrict__ b, float sign) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= N) return;
  const float l = sign * ((mR ? __ldg(mR + idx) : 0.f) - __ldg(m1 + idx));
  lam[idx] = l;
#pragma unroll
  for (int c = 0; c < 3; ++c) b[c * N + idx] = coef_b * l * __ldg(gm + c * N + idx);
}

// One backward step of the (incremental) adjoint along Y_D (Heun) fused with
// b += wb lambda_j grad m_j.
__global__ void __launch_bounds__(kT)
k3_adjoint_step(Dims d, float ht, float wb, const float* __restrict__ coef,
                const float* __restrict__ dY, const float* __restrict__ delta,
                const float* __restrict__ delta_bar, const float* __restrict__ gm,
                float* __restrict__ lam_out, float* __restrict__ b, int lagrange) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= d.N) return;
  int i, j, k;
  split3(idx, d, i, j, k);
  const long long N = d.N;
  const float db = __ldg(delta_bar + idx), dd = __ldg(delta + idx);
  const Stencil3 S = stencil3(i, j, k, __ldg(dY + idx), __ldg(dY + N + idx),
                              __ldg(dY + 2 * N + idx), d, lagrange);
  const float lb = apply3(S, coef);
  const float lstar = fmaf(ht * lb, db, lb);
  const float l = lb + 0.5f * ht * (lb * db + lstar * dd);
  lam_out[idx] = l;
#pragma unroll
  for (int c = 0; c < 3; ++c) b[c * N + idx] = fmaf(wb * l, __ldg(gm + c * N + idx), b[c * N + idx]);
}

// One forward step of the incremental state (GN):
//   m~_j = m~_{j-1}(X_D) - h_t/2 (v~(X_D) . grad m_{j-1}(X_D) + v~ . grad m_j);
// first: m~_0 = 0 and v~(X_D) gathered from cvt (written to vtD).
__global__ void __launch_bounds__(kT)
k3_incstate_step(Dims d, float ht, const float* __restrict__ coef, const float* __restrict__ dX,
                 const float* __restrict__ vt, float* __restrict__ vtD,
                 const float* __restrict__ G, const float* __restrict__ gm,
                 float* __restrict__ out, int first, const float* __restrict__ cvt,
                 int lagrange) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= d.N) return;
  int i, j, k;
  split3(idx, d, i, j, k);
  const long long N = d.N;
  const Stencil3 S = stencil3(i, j, k, __ldg(dX + idx), __ldg(dX + N + idx),
                              __ldg(dX + 2 * N + idx), d, lagrange);
  float m = first ? 0.f : apply3(S, coef);
  float w[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (first) {
      w[c] = apply3(S, cvt + c * N);
      vtD[c * N + idx] = w[c];
    } else {
      w[c] = __ldg(vtD + c * N + idx);
    }
  }
  float src = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    src += w[c] * __ldg(G + c * N + idx) + __ldg(vt + c * N + idx) * __ldg(gm + c * N + idx);
  out[idx] = m - 0.5f * ht * src;
}

// --------------------------------------------------------------------------
// Spectral multipliers (3D): real fields in and out through complex
// buffers; wavenumbers in FFT order, the Nyquist mode zeroed for the odd
// operators (grad, div); (beta |k|^2p)^s with the zero entry of |k|^2p set to
// one for s != 1 (eq. reg-precond: the mean is scaled by beta^s).
enum Op3 { OP3_GRAD = 0, OP3_DIV = 1, OP3_REGPOW = 2 };

__global__ void __launch_bounds__(kT)
k3_pack(const float* __restrict__ in, float2* __restrict__ z, long long n) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx < n) z[idx] = make_float2(__ldg(in + idx), 0.f);
}

__global__ void __launch_bounds__(kT)
k3_unpack(const float2* __restrict__ z, float* __restrict__ out, const float* __restrict__ add,
          long long n) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx < n) out[idx] = z[idx].x + (add ? __ldg(add + idx) : 0.f);
}

__device__ __forceinline__ float regpow3(float beta, int p, float s, float k2n) {
  float g = k2n;
  if (p == 2) g = k2n * k2n;
  else if (p == 3) g = k2n * k2n * k2n;
  if (s == 1.f) return beta * g;
  if (g == 0.f) g = 1.f;
  const float bg = beta * g;
  if (s == -1.f) return 1.f / bg;
  if (s == -0.5f) return 1.f / sqrtf(bg);
  if (s == 0.5f) return sqrtf(bg);
  return powf(bg, s);
}

// zout = op(zin) scaled by 1 / N (the normalisation of the inverse passes)
__global__ void __launch_bounds__(kT)
k3_multiply(Dims d, int op, int F, float beta, int p, float s, const float2* __restrict__ zin,
            float2* __restrict__ zout) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= d.N) return;
  int i, j, k;
  split3(idx, d, i, j, k);
  const long long N = d.N;
  const float scale = 1.f / (float)N;
  const float k1 = (float)signed_k(i, d.n1), k2 = (float)signed_k(j, d.n2),
              k3 = (float)signed_k(k, d.n3);
  const float q1 = (2 * i == d.n1) ? 0.f : k1, q2 = (2 * j == d.n2) ? 0.f : k2,
              q3 = (2 * k == d.n3) ? 0.f : k3;
  if (op == OP3_GRAD) {
    const float2 u = zin[idx];
    const float q[3] = {q1, q2, q3};
#pragma unroll
    for (int c = 0; c < 3; ++c)   // i q u
      zout[c * N + idx] = make_float2(-q[c] * u.y * scale, q[c] * u.x * scale);
  } else if (op == OP3_DIV) {
    const float2 a = zin[idx], b = zin[N + idx], c = zin[2 * N + idx];
    const float re = -(q1 * a.y + q2 * b.y + q3 * c.y), im = q1 * a.x + q2 * b.x + q3 * c.x;
    zout[idx] = make_float2(re * scale, im * scale);
  } else {
    const float g = regpow3(beta, p, s, k1 * k1 + k2 * k2 + k3 * k3) * scale;
    for (int c = 0; c < F; ++c) {
      const float2 u = zin[c * N + idx];
      zout[c * N + idx] = make_float2(g * u.x, g * u.y);
    }
  }
}

// Two real fields share one complex transform. The multipliers below (i q_a
// of the gradient, Nyquist zeroed, and the real even (beta |k|^2p)^s) map
// real fields to real fields, so the inverse transform of op applied to the
// spectrum of u + i w is op(u) + i op(w): half the transforms of separate
// fields, and no separation of the two spectra.

// z_p = in_{2p} + i in_{2p+1} (imaginary part 0 for the last of an odd F);
// blockIdx.y = p
__global__ void __launch_bounds__(kT)
k3_pack_pairs(const float* __restrict__ in, int F, float2* __restrict__ z, long long N) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  const int p = blockIdx.y;
  if (idx >= N) return;
  const float re = __ldg(in + 2 * p * N + idx);
  const float im = 2 * p + 1 < F ? __ldg(in + (2 * p + 1) * N + idx) : 0.f;
  z[p * N + idx] = make_float2(re, im);
}

// F output fields (+ add) from packed results, blockIdx.y = p: the real
// and imaginary parts of z_p go to out_{2p} and out_{2p+1} (interleaved,
// mode 0; no imaginary output past F) or to out_p and out_{p+H} (blocked,
// mode 1, F = 2 H)
__global__ void __launch_bounds__(kT)
k3_unpack_pairs(const float2* __restrict__ z, int mode, int H, int F, float* __restrict__ out,
                const float* __restrict__ add, long long N) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  const int p = blockIdx.y;
  if (idx >= N) return;
  const int fr = mode == 0 ? 2 * p : p, fi = mode == 0 ? 2 * p + 1 : p + H;
  const float2 v = z[p * N + idx];
  out[fr * N + idx] = v.x + (add ? __ldg(add + fr * N + idx) : 0.f);
  if (fi < F) out[fi * N + idx] = v.y + (add ? __ldg(add + fi * N + idx) : 0.f);
}

enum Op3P {
  OPP_REGPOW = 0,   // P packed spectra times (beta |k|^2p)^s
  OPP_GRAD1 = 1,    // spectrum U of one real field -> i q1 U + i (i q2 U), i q3 U
  OPP_GRAD2 = 2     // packed pair Z -> i q_c Z, c = 1, 2, 3
};

// zout = op(zin) scaled by 1 / N (the normalisation of the inverse passes)
__global__ void __launch_bounds__(kT)
k3_multiply_pairs(Dims d, int op, int P, float beta, int p, float s,
                  const float2* __restrict__ zin, float2* __restrict__ zout) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= d.N) return;
  int i, j, k;
  split3(idx, d, i, j, k);
  const long long N = d.N;
  const float scale = 1.f / (float)N;
  const float k1 = (float)signed_k(i, d.n1), k2 = (float)signed_k(j, d.n2),
              k3 = (float)signed_k(k, d.n3);
  const float q1 = (2 * i == d.n1) ? 0.f : k1, q2 = (2 * j == d.n2) ? 0.f : k2,
              q3 = (2 * k == d.n3) ? 0.f : k3;
  if (op == OPP_REGPOW) {
    const float g = regpow3(beta, p, s, k1 * k1 + k2 * k2 + k3 * k3) * scale;
    for (int c = 0; c < P; ++c) {
      const float2 u = zin[c * N + idx];
      zout[c * N + idx] = make_float2(g * u.x, g * u.y);
    }
  } else if (op == OPP_GRAD1) {
    const float2 u = zin[idx];
    // i q1 U + i (i q2 U) = (-q1 u.y - q2 u.x, q1 u.x - q2 u.y)
    zout[idx] = make_float2((-q1 * u.y - q2 * u.x) * scale, (q1 * u.x - q2 * u.y) * scale);
    zout[N + idx] = make_float2(-q3 * u.y * scale, q3 * u.x * scale);
  } else {
    const float2 u = zin[idx];
    const float q[3] = {q1, q2, q3};
#pragma unroll
    for (int c = 0; c < 3; ++c)   // i q u
      zout[c * N + idx] = make_float2(-q[c] * u.y * scale, q[c] * u.x * scale);
  }
}

// u_c += h_c dX_c (the step's own displacement, cells -> physical units)
__global__ void __launch_bounds__(kT)
k3_add_disp(long long N, float h1, float h2, float h3, const float* __restrict__ dX,
            float* __restrict__ u) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= N) return;
  u[idx] = u[idx] + h1 * __ldg(dX + idx);
  u[N + idx] = u[N + idx] + h2 * __ldg(dX + N + idx);
  u[2 * N + idx] = u[2 * N + idx] + h3 * __ldg(dX + 2 * N + idx);
}

// det (I + grad u) expanded along its first row; d12 holds grad u_1 then
// grad u_2 (six fields), d3 grad u_3 (three), field b of grad u_a = d_b u_a
__global__ void __launch_bounds__(kT)
k3_det_grad(long long N, const float* __restrict__ d12, const float* __restrict__ d3f,
            float* __restrict__ det) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= N) return;
  float J[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    J[0][b] = (b == 0 ? 1.f : 0.f) + __ldg(d12 + b * N + idx);
    J[1][b] = (b == 1 ? 1.f : 0.f) + __ldg(d12 + (3 + b) * N + idx);
    J[2][b] = (b == 2 ? 1.f : 0.f) + __ldg(d3f + b * N + idx);
  }
  det[idx] = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
             J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
             J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// ---------------------------------------------------------------------------
// Two-level preconditioner (§3.4.2) on 3D grids: spectra of the fine grid
// (n_i) and of the coarse grid (n_i / 2), P packed spectra N apart. A fine
// mode is kept by the cut-off when |k_i| < n_i / 4 on every axis: exactly the
// coarse grid's modes without its Nyquist planes. e = -1/2 multiplies by
// (beta |k|^2p)^-1/2 (the split preconditioner's factor), e = 0 by one.
__device__ __forceinline__ float split_weight(float beta, int p, float e, float k2n) {
  return e == 0.f ? 1.f : regpow3(beta, p, e, k2n);
}

// C_q = s w(k) Z_q at the coarse modes below the cut-off, 0 on the coarse
// Nyquist planes (grid over the coarse points)
__global__ void __launch_bounds__(kT)
k3_restrict_spec(Dims df, Dims dc, int P, float s, float beta, int p, float e,
                 const float2* __restrict__ Z, float2* __restrict__ C) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= dc.N) return;
  int i, j, k;
  split3(idx, dc, i, j, k);
  if (2 * i == dc.n1 || 2 * j == dc.n2 || 2 * k == dc.n3) {
    for (int q = 0; q < P; ++q) C[q * dc.N + idx] = make_float2(0.f, 0.f);
    return;
  }
  const int k1 = signed_k(i, dc.n1), k2 = signed_k(j, dc.n2), k3 = signed_k(k, dc.n3);
  const int fi = k1 < 0 ? k1 + df.n1 : k1, fj = k2 < 0 ? k2 + df.n2 : k2,
            fk = k3 < 0 ? k3 + df.n3 : k3;
  const long long fidx = ((long long)fk * df.n2 + fj) * df.n1 + fi;
  const float w = s * split_weight(beta, p, e, (float)(k1 * k1 + k2 * k2 + k3 * k3));
  for (int q = 0; q < P; ++q) {
    const float2 z = Z[q * df.N + fidx];
    C[q * dc.N + idx] = make_float2(w * z.x, w * z.y);
  }
}

// H_q = w(k) Z_q above the cut-off, 0 below (grid over the fine points)
__global__ void __launch_bounds__(kT)
k3_highpass_spec(Dims df, int P, float beta, int p, float e, const float2* __restrict__ Z,
                 float2* __restrict__ H) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= df.N) return;
  int i, j, k;
  split3(idx, df, i, j, k);
  const int k1 = signed_k(i, df.n1), k2 = signed_k(j, df.n2), k3 = signed_k(k, df.n3);
  const bool kept = 4 * abs(k1) < df.n1 && 4 * abs(k2) < df.n2 && 4 * abs(k3) < df.n3;
  const float w = kept ? 0.f : split_weight(beta, p, e, (float)(k1 * k1 + k2 * k2 + k3 * k3));
  for (int q = 0; q < P; ++q) {
    const float2 z = Z[q * df.N + idx];
    H[q * df.N + idx] = make_float2(w * z.x, w * z.y);
  }
}

// out_q = w(k) (sc Sc_q[coarse(k)] below the cut-off, sh H_q above; H may be
// NULL: 0) on the fine grid: prolongation by zero padding plus the high band
__global__ void __launch_bounds__(kT)
k3_prolong_spec(Dims df, Dims dc, int P, float sc, const float2* __restrict__ Sc, float sh,
                const float2* __restrict__ H, float beta, int p, float e,
                float2* __restrict__ out) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= df.N) return;
  int i, j, k;
  split3(idx, df, i, j, k);
  const int k1 = signed_k(i, df.n1), k2 = signed_k(j, df.n2), k3 = signed_k(k, df.n3);
  const bool kept = 4 * abs(k1) < df.n1 && 4 * abs(k2) < df.n2 && 4 * abs(k3) < df.n3;
  const float w = split_weight(beta, p, e, (float)(k1 * k1 + k2 * k2 + k3 * k3));
  long long cidx = 0;
  if (kept) {
    const int ci = k1 < 0 ? k1 + dc.n1 : k1, cj = k2 < 0 ? k2 + dc.n2 : k2,
              ck = k3 < 0 ? k3 + dc.n3 : k3;
    cidx = ((long long)ck * dc.n2 + cj) * dc.n1 + ci;
  }
  for (int q = 0; q < P; ++q) {
    float2 z = make_float2(0.f, 0.f);
    if (kept) {
      const float2 c = Sc[q * dc.N + cidx];
      z = make_float2(sc * c.x, sc * c.y);
    } else if (H) {
      const float2 h = H[q * df.N + idx];
      z = make_float2(sh * h.x, sh * h.y);
    }
    out[q * df.N + idx] = make_float2(w * z.x, w * z.y);
  }
}

// z = a + i b for two separate real fields; a = Re z, b = Im z back
__global__ void __launch_bounds__(kT)
k3_pack_two(const float* __restrict__ a, const float* __restrict__ b, float2* __restrict__ z,
            long long N) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx < N) z[idx] = make_float2(__ldg(a + idx), __ldg(b + idx));
}

__global__ void __launch_bounds__(kT)
k3_unpack_two(const float2* __restrict__ z, float* __restrict__ a, float* __restrict__ b,
              long long N) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
  if (idx >= N) return;
  const float2 v = z[idx];
  a[idx] = v.x;
  b[idx] = v.y;
}

inline unsigned nb(long long n) { return (unsigned)((n + kT - 1) / kT); }

}  // namespace d3
}  // namespace regnk

using namespace regnk;
using namespace regnk::d3;

struct reg3_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  reg_options opt;
  Dims d{};
  int nt = 0;
  float ht = 0.f;
  double beta = 0, hh = 0;
  bool lagrange = false;
  float s1 = 0, s2 = 0, s3 = 0;
  float2 *tw1 = nullptr, *tw2 = nullptr, *tw3 = nullptr;
  float *mR = nullptr, *mT = nullptr, *v = nullptr, *cv = nullptr, *dX = nullptr, *dY = nullptr,
        *delta = nullptr, *delta_bar = nullptr, *m = nullptr, *gm = nullptr, *G = nullptr,
        *coef = nullptr, *c3 = nullptr, *tA = nullptr, *fA = nullptr,
        *fB = nullptr, *vtD = nullptr, *b = nullptr, *Av = nullptr;
  float *kx = nullptr, *kr = nullptr, *kz = nullptr, *kp = nullptr, *kq = nullptr,
        *vtrial = nullptr, *gcur = nullptr, *rhs = nullptr;
  float2 *zA = nullptr, *zB = nullptr;
  double* partial = nullptr;
  float* partialf = nullptr;
  double* dsc = nullptr;
  double* hsc = nullptr;
  int* dflag = nullptr;
  int* hflag = nullptr;
  bool have_images = false, have_v = false, have_G = false;
  // shared-memory boxes of the gathers along X_D, Y_D and of the departure
  // kernel (reach s v); use_* false: the global-load kernels
  bool boxes = true;
  Box3 boxX{}, boxY{}, boxV{};
  bool useX = false, useY = false, useV = false;
  // P_2L (§3.4.2): the coarse problem on the grid of n_i / 2 points (its own
  // context), the Chebyshev bounds of its split operator and coarse-grid
  // work vectors (three fields each)
  reg3_ctx* coarse = nullptr;
  double emin = 0, emax = 0;
  bool have_eig = false;
  int coarse_matvecs = 0;
  double eta = 0.5;   // forcing term of the Newton step (PCG(eps eta) coarse solves)
  float *pc_rc = nullptr, *pc_sc = nullptr, *pc_r = nullptr, *pc_d = nullptr, *pc_w = nullptr,
        *pc_u = nullptr, *pc_q = nullptr, *pc_v = nullptr;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

struct D3Error {
  reg_status s;
};

void fail(reg3_ctx* c, reg_status s, const std::string& msg) {
  c->err = msg;
  throw D3Error{s};
}

void check(reg3_ctx* c, cudaError_t e, const char* what) {
  if (e != cudaSuccess)
    fail(c, e == cudaErrorMemoryAllocation ? REG_ENOMEM : REG_ECUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
}

void check_launch(reg3_ctx* c, const char* what) { check(c, cudaGetLastError(), what); }

template <typename T>
T* dalloc(reg3_ctx* c, size_t n) {
  void* p = nullptr;
  check(c, cudaMalloc(&p, n * sizeof(T) + 16), "cudaMalloc");
  c->allocs.push_back(p);
  return static_cast<T*>(p);
}

float2* twiddles(reg3_ctx* c, int n) {
  std::vector<float2> h(n);
  for (int k = 0; k < n; ++k) {
    const double a = -2.0 * M_PI * (double)k / (double)n;
    h[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  float2* d = dalloc<float2>(c, n);
  check(c, cudaMemcpy(d, h.data(), n * sizeof(float2), cudaMemcpyHostToDevice), "twiddles");
  return d;
}

// the three axis passes of a 3D FFT of F complex arrays in z
void fft3(reg3_ctx* c, float2* z, int F, bool inverse) {
  const Dims& d = c->d;
  fft_axis(z, d.N, F, d.n1, 1, inverse, c->tw1, c->st);
  fft_axis(z, d.N, F, d.n2, d.n1, inverse, c->tw2, c->st);
  fft_axis(z, d.N, F, d.n3, (long long)d.n1 * d.n2, inverse, c->tw3, c->st);
}

// out (Fout fields) = op(in (Fin fields)) [+ add]
void spectral3(reg3_ctx* c, int op, double s, const float* in, int Fin, float* out, int Fout,
               const float* add) {
  const long long N = c->d.N;
  if (op == OP3_DIV) {   // 3 -> 1: three separate spectra
    launch_k(k3_pack, dim3(nb(Fin * N)), dim3(kT), 0, c->st, in, c->zA, Fin * N);
    fft3(c, c->zA, Fin, false);
    launch_k(k3_multiply, dim3(nb(N)), dim3(kT), 0, c->st, c->d, op, Fin, (float)c->beta,
             c->opt.reg_norm, (float)s, (const float2*)c->zA, c->zB);
    fft3(c, c->zB, Fout, true);
    launch_k(k3_unpack, dim3(nb(Fout * N)), dim3(kT), 0, c->st, (const float2*)c->zB, out, add,
             Fout * N);
  } else {   // grad (1 -> 3) or (beta A)^s (F -> F) on packed pairs
    const int Pin = (Fin + 1) / 2, Pout = (Fout + 1) / 2;
    launch_k(k3_pack_pairs, dim3(nb(N), Pin), dim3(kT), 0, c->st, in, Fin, c->zA, N);
    fft3(c, c->zA, Pin, false);
    launch_k(k3_multiply_pairs, dim3(nb(N)), dim3(kT), 0, c->st, c->d,
             op == OP3_GRAD ? (int)OPP_GRAD1 : (int)OPP_REGPOW, Pin, (float)c->beta,
             c->opt.reg_norm, (float)s, (const float2*)c->zA, c->zB);
    fft3(c, c->zB, Pout, true);
    launch_k(k3_unpack_pairs, dim3(nb(N), Pout), dim3(kT), 0, c->st, (const float2*)c->zB, 0, 0,
             Fout, out, add, N);
  }
  check_launch(c, "spectral operator");
}

// the gradients of the two consecutive fields u and u + N into out (the three
// components of the first, then those of the second) with one forward and
// three inverse transforms
void grad_pair(reg3_ctx* c, const float* u, float* out) {
  const long long N = c->d.N;
  launch_k(k3_pack_pairs, dim3(nb(N), 1), dim3(kT), 0, c->st, u, 2, c->zA, N);
  fft3(c, c->zA, 1, false);
  launch_k(k3_multiply_pairs, dim3(nb(N)), dim3(kT), 0, c->st, c->d, (int)OPP_GRAD2, 1,
           (float)c->beta, c->opt.reg_norm, 0.f, (const float2*)c->zA, c->zB);
  fft3(c, c->zB, 3, true);
  launch_k(k3_unpack_pairs, dim3(nb(N), 3), dim3(kT), 0, c->st, (const float2*)c->zB, 1, 3, 6, out,
           (const float*)nullptr, N);
  check_launch(c, "gradient pair");
}

// interpolation coefficients of F consecutive fields (the samples themselves
// for cubic Lagrange)
const float* coefficients(reg3_ctx* c, const float* u, int F, float* dst) {
  if (c->lagrange) return u;
  const Dims& d = c->d;
  // x_1 pass into dst, x_2 pass dst -> tA, x_3 pass tA -> dst (F fields each)
  launch_k(k3_prefilter_lines<0>, dim3((unsigned)(d.N / d.n1 / 32), F), dim3(d.n1),
           (size_t)32 * (d.n1 + 1) * sizeof(float), c->st, u, dst, d);
  launch_k(k3_prefilter_lines<1>, dim3((unsigned)(d.n1 / 32 * d.n3), F), dim3(d.n2),
           (size_t)32 * d.n2 * sizeof(float), c->st, (const float*)dst, c->tA, d);
  launch_k(k3_prefilter_lines<2>, dim3((unsigned)(d.n1 / 32 * d.n2), F), dim3(d.n3),
           (size_t)32 * d.n3 * sizeof(float), c->st, (const float*)c->tA, dst, d);
  check_launch(c, "prefilter");
  return dst;
}

// box of a gather whose displacements are bounded by D_a cells per axis;
// false when it does not fit (the global-load kernels run instead)
constexpr size_t kBoxMaxBytes = 112 * 1024;

bool make_box(const reg3_ctx* c, const double D[3], Box3& g) {
  int lo[3], hi[3];
  const int n[3] = {c->d.n1, c->d.n2, c->d.n3};
  for (int a = 0; a < 3; ++a) {
    if (!(D[a] >= 0.0) || D[a] > 64.0) return false;   // NaN, or far outside any box
    lo[a] = (int)std::ceil(D[a]) + 1;
    hi[a] = (int)std::floor(D[a]) + 2;
    if (lo[a] >= n[a] || hi[a] >= n[a]) return false;
  }
  g = Box3{lo[0], lo[1], lo[2], kBX + lo[0] + hi[0], kBY + lo[1] + hi[1], kBZ + lo[2] + hi[2]};
  return g.b1 <= kBoxPitch && (size_t)kBoxPitch * g.b2 * g.b3 * sizeof(float) <= kBoxMaxBytes;
}

size_t box_bytes(const Box3& g) { return (size_t)kBoxPitch * g.b2 * g.b3 * sizeof(float); }

unsigned box_blocks(const Dims& d) { return (unsigned)((d.n1 / kBX) * (d.n2 / kBY) * (d.n3 / kBZ)); }

// max |u_a| of the three components of a vector field, to the host
void max3(reg3_ctx* c, const float* u, double out[3]) {
  const long long N = c->d.N;
  for (int a = 0; a < 3; ++a) launch_maxabs(u + a * N, N, c->partialf, c->dsc + a, c->st);
  check(c, cudaMemcpyAsync(c->hsc, c->dsc, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->st), "read");
  check(c, cudaStreamSynchronize(c->st), "synchronize");
  for (int a = 0; a < 3; ++a) out[a] = c->hsc[a];
}

// the box of the gathers along disp (X_D or Y_D of the cached velocity)
bool box_for(const reg3_ctx* c, const float* disp, Box3& g) {
  if (disp == c->dX && c->useX) { g = c->boxX; return true; }
  if (disp == c->dY && c->useY) { g = c->boxY; return true; }
  return false;
}

void gather(reg3_ctx* c, const float* u, int F, const float* disp, float* out, float* cbuf) {
  const float* cu = coefficients(c, u, F, cbuf);
  Box3 g;
  if (box_for(c, disp, g))
    launch_k(k3b_gather, dim3(box_blocks(c->d)), dim3(kBT), box_bytes(g), c->st, c->d, g, cu, disp,
             out, F, (int)c->lagrange);
  else
    launch_k(k3_gather, dim3(nb(c->d.N)), dim3(kT), 0, c->st, c->d, cu, disp, out, F, (int)c->lagrange);
  check_launch(c, "gather");
}

// departure points X_D, Y_D of c->v (coefficients cv) and the boxes of the
// gathers along them
void departure(reg3_ctx* c, const float* cv) {
  const long long N = c->d.N;
  c->useV = c->useX = c->useY = false;
  if (c->boxes) {
    double vm[3];
    max3(c, c->v, vm);
    // the reach |s_a v_a| of the first Heun stage, with a margin for the
    // FP32 product
    const double D[3] = {vm[0] * c->s1 * (1.0 + 1e-5), vm[1] * c->s2 * (1.0 + 1e-5),
                         vm[2] * c->s3 * (1.0 + 1e-5)};
    c->useV = make_box(c, D, c->boxV);
  }
  if (c->useV)
    launch_k(k3b_departure, dim3(box_blocks(c->d)), dim3(kBT), box_bytes(c->boxV), c->st, c->d,
             c->boxV, c->s1, c->s2, c->s3, (const float*)c->v, cv, c->dX, c->dY, (int)c->lagrange);
  else
    launch_k(k3_departure, dim3(nb(N)), dim3(kT), 0, c->st, c->d, c->s1, c->s2, c->s3,
             (const float*)c->v, cv, c->dX, c->dY, (int)c->lagrange);
  check_launch(c, "departure");
  if (c->boxes) {
    double DX[3], DY[3];
    max3(c, c->dX, DX);
    max3(c, c->dY, DY);
    c->useX = make_box(c, DX, c->boxX);
    c->useY = make_box(c, DY, c->boxY);
  }
}

// v, its characteristics, the state history m_0..m_nt, grad m_j, div v and
// div v at Y_D (§3.3.2)
void set_velocity(reg3_ctx* c, const float* v) {
  const long long N = c->d.N;
  const int nt = c->nt;
  if (v != c->v)
    check(c, cudaMemcpyAsync(c->v, v, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy v");
  departure(c, coefficients(c, c->v, 3, c->cv));
  check(c, cudaMemcpyAsync(c->m, c->mT, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "m_T");
  for (int j = 1; j <= nt; ++j) gather(c, c->m + (j - 1) * N, 1, c->dX, c->m + j * N, c->coef);
  int j = 0;
  for (; j + 1 <= nt; j += 2) grad_pair(c, c->m + j * N, c->gm + 3 * j * N);
  if (j == nt) spectral3(c, OP3_GRAD, 0.0, c->m + j * N, 1, c->gm + 3 * j * N, 3, nullptr);
  spectral3(c, OP3_DIV, 0.0, c->v, 3, c->delta, 1, nullptr);
  gather(c, c->delta, 1, c->dY, c->delta_bar, c->coef);
  c->have_v = true;
  c->have_G = false;
}

// set_velocity unless v equals the cached velocity bit for bit (a device
// compare and one synchronisation)
void sync_velocity(reg3_ctx* c, const float* v) {
  bool differ = true;
  if (c->have_v) {
    check(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st), "memset");
    launch_compare(v, c->v, 3 * c->d.N, c->dflag, c->st);
    check(c, cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->st), "flag");
    check(c, cudaStreamSynchronize(c->st), "synchronize");
    differ = (*c->hflag != 0);
  }
  if (differ) set_velocity(c, v);
}

void ensure_G(reg3_ctx* c) {
  if (c->have_G) return;
  const long long N = c->d.N;
  for (int j = 1; j <= c->nt; ++j)
    gather(c, c->gm + 3 * (j - 1) * N, 3, c->dX, c->G + 3 * (j - 1) * N, c->c3);
  c->have_G = true;
}

double dot_sync(reg3_ctx* c, const float* a, const float* b, long long n) {
  launch_dot(a, b, n, c->partial, c->dsc, c->st);
  check(c, cudaMemcpyAsync(c->hsc, c->dsc, sizeof(double), cudaMemcpyDeviceToHost, c->st), "read");
  check(c, cudaStreamSynchronize(c->st), "synchronize");
  return c->hsc[0];
}

// J = 1/2 <m_1 - m_R, m_1 - m_R>_h + beta/2 <v, A v>_h; leaves beta A v in Av
double objective(reg3_ctx* c) {
  const long long N = c->d.N;
  spectral3(c, OP3_REGPOW, 1.0, c->v, 3, c->Av, 3, nullptr);
  launch_sumsq_diff(c->m + c->nt * N, c->mR, N, c->partial, c->dsc, c->st);
  launch_dot(c->v, c->Av, 3 * N, c->partial, c->dsc + 1, c->st);
  check(c, cudaMemcpyAsync(c->hsc, c->dsc, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st), "read");
  check(c, cudaStreamSynchronize(c->st), "synchronize");
  return 0.5 * c->hh * c->hsc[0] + 0.5 * c->hh * c->hsc[1];
}

// one backward (incremental) adjoint step along Y_D from the coefficients cl
void adjoint_step(reg3_ctx* c, const float* cl, float wb, const float* gmj, float* lam_out) {
  if (c->useY)
    launch_k(k3b_adjoint_step, dim3(box_blocks(c->d)), dim3(kBT), box_bytes(c->boxY), c->st, c->d,
             c->boxY, c->ht, wb, cl, (const float*)c->dY, (const float*)c->delta,
             (const float*)c->delta_bar, gmj, lam_out, c->b, (int)c->lagrange);
  else
    launch_k(k3_adjoint_step, dim3(nb(c->d.N)), dim3(kT), 0, c->st, c->d, c->ht, wb, cl,
             (const float*)c->dY, (const float*)c->delta, (const float*)c->delta_bar, gmj, lam_out,
             c->b, (int)c->lagrange);
}

// one forward incremental state step along X_D (first: m~_0 = 0 and v~(X_D)
// gathered from cvt into vtD)
void incstate_step(reg3_ctx* c, const float* cm, const float* vt, const float* Gj,
                   const float* gmj, float* out, bool first, const float* cvt) {
  if (c->useX)
    launch_k(k3b_incstate_step, dim3(box_blocks(c->d)), dim3(kBT), box_bytes(c->boxX), c->st, c->d,
             c->boxX, c->ht, cm, (const float*)c->dX, vt, c->vtD, Gj, gmj, out, (int)first, cvt,
             (int)c->lagrange);
  else
    launch_k(k3_incstate_step, dim3(nb(c->d.N)), dim3(kT), 0, c->st, c->d, c->ht, cm,
             (const float*)c->dX, vt, c->vtD, Gj, gmj, out, (int)first, cvt, (int)c->lagrange);
}

// g = beta A v + int_0^1 lambda grad m dt (eq. control-elim, K = I)
void gradient(reg3_ctx* c, float* g) {
  const long long N = c->d.N;
  const int nt = c->nt;
  const float ht = c->ht;
  float* lam = c->fA;
  float* lam2 = c->fB;
  launch_k(k3_adjoint_init, dim3(nb(N)), dim3(kT), 0, c->st, N, 0.5f * ht, (const float*)c->mR,
           (const float*)(c->m + nt * N), (const float*)(c->gm + 3 * nt * N), lam, c->b, 1.f);
  for (int j = nt - 1; j >= 0; --j) {
    const float wb = ht * (j == 0 ? 0.5f : 1.0f);
    adjoint_step(c, coefficients(c, lam, 1, c->coef), wb, c->gm + 3 * j * N, lam2);
    std::swap(lam, lam2);
  }
  launch_lincomb(3 * N, 1.f, c->Av, 1.f, c->b, g, c->st);
  check_launch(c, "gradient");
}

// Gauss-Newton H v~ = beta A v~ + int lambda~ grad m dt (eq. hessian-matvec);
// data_only: the data term int lambda~ grad m dt alone
void hessian(reg3_ctx* c, const float* vt, float* out, bool data_only = false) {
  const long long N = c->d.N;
  const int nt = c->nt;
  const float ht = c->ht;
  ensure_G(c);
  const float* cvt = coefficients(c, vt, 3, c->c3);
  float* mt = c->fA;
  float* mt2 = c->fB;
  for (int j = 1; j <= nt; ++j) {
    const float* cm = j == 1 ? nullptr : coefficients(c, mt, 1, c->coef);
    incstate_step(c, cm, vt, c->G + 3 * (j - 1) * N, c->gm + 3 * j * N, mt2, j == 1, cvt);
    std::swap(mt, mt2);
  }
  // lambda~_nt = -m~_nt and the first term of the time integral
  launch_k(k3_adjoint_init, dim3(nb(N)), dim3(kT), 0, c->st, N, 0.5f * ht, (const float*)nullptr,
           (const float*)mt, (const float*)(c->gm + 3 * nt * N), mt2, c->b, 1.f);
  float* lt = mt2;
  float* lt2 = mt;
  for (int j = nt - 1; j >= 0; --j) {
    const float wb = ht * (j == 0 ? 0.5f : 1.0f);
    adjoint_step(c, coefficients(c, lt, 1, c->coef), wb, c->gm + 3 * j * N, lt2);
    std::swap(lt, lt2);
  }
  if (data_only)
    check(c, cudaMemcpyAsync(out, c->b, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  else
    spectral3(c, OP3_REGPOW, 1.0, vt, 3, out, 3, c->b);
  check_launch(c, "hessian");
}

// -- two-level preconditioner --------------------------------------------------
// the three components of a fine-grid vector field restricted to the coarse
// grid (§3.4.2): one fine transform, the kept modes copied, one coarse
// transform
void restrict_to_coarse(reg3_ctx* c, const float* in, float* out) {
  reg3_ctx* cc = c->coarse;
  const long long Nf = c->d.N, Nc = cc->d.N;
  launch_k(k3_pack_pairs, dim3(nb(Nf), 2), dim3(kT), 0, c->st, in, 3, c->zA, Nf);
  fft3(c, c->zA, 2, false);
  launch_k(k3_restrict_spec, dim3(nb(Nc)), dim3(kT), 0, c->st, c->d, cc->d, 2, 1.f / (float)Nf, 0.f,
           0, 0.f, (const float2*)c->zA, cc->zB);
  fft3(cc, cc->zB, 2, true);
  launch_k(k3_unpack_pairs, dim3(nb(Nc), 2), dim3(kT), 0, c->st, (const float2*)cc->zB, 0, 0, 3, out,
           (const float*)nullptr, Nc);
  check_launch(c, "restriction");
}

void restrict_images(reg3_ctx* c) {
  reg3_ctx* cc = c->coarse;
  const long long Nf = c->d.N, Nc = cc->d.N;
  launch_k(k3_pack_two, dim3(nb(Nf)), dim3(kT), 0, c->st, (const float*)c->mR, (const float*)c->mT,
           c->zA, Nf);
  fft3(c, c->zA, 1, false);
  launch_k(k3_restrict_spec, dim3(nb(Nc)), dim3(kT), 0, c->st, c->d, cc->d, 1, 1.f / (float)Nf, 0.f,
           0, 0.f, (const float2*)c->zA, cc->zB);
  fft3(cc, cc->zB, 1, true);
  launch_k(k3_unpack_two, dim3(nb(Nc)), dim3(kT), 0, c->st, (const float2*)cc->zB, cc->mR, cc->mT, Nc);
  check_launch(c, "restriction");
  cc->have_images = true;
  cc->have_v = cc->have_G = false;
}

// out = (I + (beta A_c)^-1/2 Q_c (beta A_c)^-1/2) s on the coarse grid
void coarse_split(reg3_ctx* c, const float* s, float* out) {
  reg3_ctx* cc = c->coarse;
  spectral3(cc, OP3_REGPOW, -0.5, s, 3, c->pc_u, 3, nullptr);
  hessian(cc, c->pc_u, c->pc_q, true);
  spectral3(cc, OP3_REGPOW, -0.5, c->pc_q, 3, out, 3, s);
  ++c->coarse_matvecs;
}

// CHEB(k) with the bounds [emin, emax] on the coarse split operator, from
// x = 0: the three-term Chebyshev iteration (k updates, k - 1 operator
// applications)
void cheb(reg3_ctx* c, const float* b, float* x) {
  const long long n = 3 * c->coarse->d.N;
  const double theta = 0.5 * (c->emax + c->emin), delta = 0.5 * (c->emax - c->emin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  check(c, cudaMemcpyAsync(c->pc_r, b, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  launch_lincomb(n, (float)(1.0 / theta), b, 0.f, nullptr, c->pc_d, c->st);
  launch_fill(x, n, 0.f, c->st);
  const int k = c->opt.cheb_iters;
  for (int it = 0; it < k; ++it) {
    launch_lincomb(n, 1.f, x, 1.f, c->pc_d, x, c->st);
    if (it == k - 1) break;
    coarse_split(c, c->pc_d, c->pc_w);
    launch_lincomb(n, 1.f, c->pc_r, -1.f, c->pc_w, c->pc_r, c->st);
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    launch_lincomb(n, (float)(rho_new * rho), c->pc_d, (float)(2.0 * rho_new / delta), c->pc_r,
                   c->pc_d, c->st);
    rho = rho_new;
  }
}

// PCG(rtol) without preconditioner on the coarse split operator from x = 0
// (the steps of the outer PCG: stop at ||r|| <= rtol ||b||, keep the
// current iterate at a non-positive curvature, b itself at the first step)
void coarse_pcg(reg3_ctx* c, const float* b, float* x, double rtol) {
  reg3_ctx* cc = c->coarse;
  const long long n = 3 * cc->d.N;
  launch_fill(x, n, 0.f, c->st);
  const double bnorm = std::sqrt(dot_sync(cc, b, b, n));
  if (!(bnorm > 0.0)) return;
  float* r = c->pc_r;
  float* p = c->pc_d;
  float* q = c->pc_w;
  check(c, cudaMemcpyAsync(r, b, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  check(c, cudaMemcpyAsync(p, b, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  double rz = bnorm * bnorm;
  for (int it = 0; it < c->opt.max_pcg; ++it) {
    coarse_split(c, p, q);
    const double pq = dot_sync(cc, p, q, n);
    if (!(pq > 0.0)) {
      if (it == 0)
        check(c, cudaMemcpyAsync(x, b, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
      break;
    }
    const float alpha = (float)(rz / pq);
    launch_lincomb(n, 1.f, x, alpha, p, x, c->st);
    launch_lincomb(n, 1.f, r, -alpha, q, r, c->st);
    const double rr = dot_sync(cc, r, r, n);
    if (std::sqrt(rr) / bnorm <= rtol) break;
    launch_lincomb(n, 1.f, r, (float)(rr / rz), p, p, c->st);
    rz = rr;
  }
}

// largest eigenvalue of the symmetric tridiagonal matrix (diagonal a,
// off-diagonal b) by bisection on the Sturm sequence count
double tridiag_largest(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  if (m == 0) return 0.0;
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  auto below = [&](double x) {   // number of eigenvalues below x
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
      q = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      cnt += q < 0.0;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::fmax(1.0, std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) == m) hi = mid; else lo = mid;
  }
  return hi;
}

// Chebyshev bounds of the coarse split operator at v = 0 (§3.4.2 "Eigenvalue
// Estimates"): e_max from lanczos_steps Lanczos steps (FP32 vectors, FP64
// inner products, SplitMix64 start vector of lanczos_seed) times
// emax_safety; e_min = min over the coarse modes of 1 + 1/(beta gamma_k)
void estimate_eig(reg3_ctx* c) {
  reg3_ctx* cc = c->coarse;
  const long long n = 3 * cc->d.N;
  launch_fill(c->pc_v, n, 0.f, c->st);
  set_velocity(cc, c->pc_v);
  float* q = c->pc_r;
  float* qprev = c->pc_d;
  float* w = c->pc_w;
  launch_splitmix(q, n, c->opt.lanczos_seed, c->st);
  const double nq = std::sqrt(dot_sync(cc, q, q, n));
  launch_lincomb(n, (float)(1.0 / nq), q, 0.f, nullptr, q, c->st);
  launch_fill(qprev, n, 0.f, c->st);
  std::vector<double> al, be;
  double beta = 0.0;
  for (int k = 0; k < c->opt.lanczos_steps; ++k) {
    coarse_split(c, q, w);
    const double alpha = dot_sync(cc, q, w, n);
    launch_lincomb(n, 1.f, w, (float)-alpha, q, w, c->st);
    launch_lincomb(n, 1.f, w, (float)-beta, qprev, w, c->st);
    al.push_back(alpha);
    const double bn = std::sqrt(dot_sync(cc, w, w, n));
    if (!(bn > 1e-12 * std::fabs(alpha))) break;
    be.push_back(bn);
    std::swap(qprev, q);
    launch_lincomb(n, (float)(1.0 / bn), w, 0.f, nullptr, q, c->st);
    beta = bn;
  }
  be.resize(al.empty() ? 0 : al.size() - 1);
  const double kn = 0.25 * ((double)cc->d.n1 * cc->d.n1 + (double)cc->d.n2 * cc->d.n2 +
                            (double)cc->d.n3 * cc->d.n3);
  c->emin = 1.0 + 1.0 / (c->beta * std::pow(kn, c->opt.reg_norm));
  c->emax = tridiag_largest(al, be) * c->opt.emax_safety;
  c->have_eig = true;
}

// the coarse problem at the restriction of v
void set_velocity_coarse(reg3_ctx* c, const float* v) {
  restrict_to_coarse(c, v, c->pc_v);
  set_velocity(c->coarse, c->pc_v);
}

// z = P_2L^-1 r: one fine transform of r, the high band kept in spectral form
// while CHEB(k) or PCG(eps eta) solves the coarse split system for the low
// band, then one
// fine transform of (beta A)^-1/2 (P s_c + H r'), r' = (beta A)^-1/2 r
void precond_2l(reg3_ctx* c, const float* r, float* z) {
  reg3_ctx* cc = c->coarse;
  const long long Nf = c->d.N, Nc = cc->d.N;
  const float b = (float)c->beta;
  const int p = c->opt.reg_norm;
  launch_k(k3_pack_pairs, dim3(nb(Nf), 2), dim3(kT), 0, c->st, r, 3, c->zA, Nf);
  fft3(c, c->zA, 2, false);
  launch_k(k3_restrict_spec, dim3(nb(Nc)), dim3(kT), 0, c->st, c->d, cc->d, 2, 1.f / (float)Nf, b, p,
           -0.5f, (const float2*)c->zA, cc->zB);
  launch_k(k3_highpass_spec, dim3(nb(Nf)), dim3(kT), 0, c->st, c->d, 2, b, p, -0.5f,
           (const float2*)c->zA, c->zB);
  fft3(cc, cc->zB, 2, true);
  launch_k(k3_unpack_pairs, dim3(nb(Nc), 2), dim3(kT), 0, c->st, (const float2*)cc->zB, 0, 0, 3,
           c->pc_rc, (const float*)nullptr, Nc);
  if (c->opt.pc_solver == REG_PCSOLVER_PCG)
    coarse_pcg(c, c->pc_rc, c->pc_sc, c->opt.pc_eps * c->eta);
  else
    cheb(c, c->pc_rc, c->pc_sc);
  launch_k(k3_pack_pairs, dim3(nb(Nc), 2), dim3(kT), 0, c->st, (const float*)c->pc_sc, 3, cc->zA, Nc);
  fft3(cc, cc->zA, 2, false);
  launch_k(k3_prolong_spec, dim3(nb(Nf)), dim3(kT), 0, c->st, c->d, cc->d, 2, 1.f / (float)Nc,
           (const float2*)cc->zA, 1.f / (float)Nf, (const float2*)c->zB, b, p, -0.5f, c->zA);
  fft3(c, c->zA, 2, true);
  launch_k(k3_unpack_pairs, dim3(nb(Nf), 2), dim3(kT), 0, c->st, (const float2*)c->zA, 0, 0, 3, z,
           (const float*)nullptr, Nf);
  check_launch(c, "P_2L");
}

// the configured preconditioner inverse
void precond(reg3_ctx* c, const float* r, float* z) {
  if (c->coarse)
    precond_2l(c, r, z);
  else
    spectral3(c, OP3_REGPOW, -1.0, r, 3, z, 3, nullptr);
}

bool size_ok3(int n) { return n % 32 == 0 && fft_axis_supported(n); }
bool unaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

reg_status guarded(reg3_ctx* c, const std::function<void()>& body) {
  if (!c) return REG_EINVAL;
  const int saved = t_programmatic_launch;
  const int saved_prec = t_plain_fp32_reduce;
  t_programmatic_launch = c->opt.programmatic_launch ? 1 : 0;
  t_plain_fp32_reduce = 0;
  reg_status s = REG_OK;
  try {
    body();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      c->err = std::string("CUDA: ") + cudaGetErrorString(e);
      s = REG_ECUDA;
    }
  } catch (const D3Error& e) {
    s = e.s;
    if (c->coarse && !c->coarse->err.empty()) {
      c->err = "coarse grid: " + c->coarse->err;
      c->coarse->err.clear();
    }
  }
  t_programmatic_launch = saved;
  t_plain_fp32_reduce = saved_prec;
  return s;
}

}  // namespace

extern "C" {

reg_status reg3_create(int n1, int n2, int n3, int nt, double beta, const reg_options* opt,
                       reg3_ctx** out) {
  if (!out) return REG_EINVAL;
  *out = nullptr;
  if (!size_ok3(n1) || !size_ok3(n2) || !size_ok3(n3) || nt < 1 || nt > 4096 || !(beta > 0.0))
    return REG_EINVAL;
  reg_options o;
  if (opt) o = *opt; else reg_default_options(&o);
  const bool two_level = o.precond == REG_PC_2L;
  if (two_level &&
      (!size_ok3(n1 / 2) || !size_ok3(n2 / 2) || !size_ok3(n3 / 2) || n1 % 2 || n2 % 2 || n3 % 2 ||
       (o.pc_solver != REG_PCSOLVER_CHEB && o.pc_solver != REG_PCSOLVER_PCG) ||
       (o.pc_solver == REG_PCSOLVER_PCG && !(o.pc_eps > 0.0)) || o.cheb_iters < 1 ||
       o.lanczos_steps < 1 ||
       !(o.emax_safety >= 1.0) || (o.coarse_nt != 0 && o.coarse_nt != nt) ||
       (o.coarse_interp != -1 && o.coarse_interp != o.interp)))
    return REG_EINVAL;
  if (o.reg_norm < 1 || o.reg_norm > 3 || (o.interp != 0 && o.interp != 1) ||
      (o.precond != REG_PC_REG && !two_level) || o.hessian != REG_HESSIAN_GN || o.incompressible ||
      o.beta_w != 0.0 || o.max_pcg < 1 || o.max_newton < 0 || o.max_backtracks < 0)
    return REG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return REG_ECUDA;
  reg3_ctx* c = new reg3_ctx();
  c->device = dev;
  c->opt = o;
  c->d = Dims{n1, n2, n3, (long long)n1 * n2 * n3};
  c->nt = nt;
  c->ht = 1.0f / (float)nt;
  c->beta = beta;
  c->hh = (2.0 * M_PI / n1) * (2.0 * M_PI / n2) * (2.0 * M_PI / n3);
  c->lagrange = (o.interp == REG_INTERP_LAGRANGE);
  c->s1 = departure_scale(c->ht, n1);
  c->s2 = departure_scale(c->ht, n2);
  c->s3 = departure_scale(c->ht, n3);
  const reg_status s = guarded(c, [&] {
    const size_t N = (size_t)c->d.N;
    c->tw1 = twiddles(c, n1);
    c->tw2 = twiddles(c, n2);
    c->tw3 = twiddles(c, n3);
    float** scalar[] = {&c->mR, &c->mT, &c->delta, &c->delta_bar, &c->coef, &c->fA, &c->fB};
    for (float** f : scalar) *f = dalloc<float>(c, N);
    float** vec[] = {&c->v, &c->cv, &c->dX, &c->dY, &c->c3, &c->tA, &c->vtD, &c->b, &c->Av, &c->kx,
                     &c->kr, &c->kz, &c->kp, &c->kq, &c->vtrial, &c->gcur, &c->rhs};
    for (float** f : vec) *f = dalloc<float>(c, 3 * N);
    c->m = dalloc<float>(c, (size_t)(nt + 1) * N);
    c->gm = dalloc<float>(c, 3 * (size_t)(nt + 1) * N);
    c->G = dalloc<float>(c, 3 * (size_t)nt * N);
    c->zA = dalloc<float2>(c, 3 * N);
    c->zB = dalloc<float2>(c, 3 * N);
    c->partial = dalloc<double>(c, reduce_partials());
    c->partialf = dalloc<float>(c, reduce_partials());
    c->dsc = dalloc<double>(c, 4);
    c->dflag = dalloc<int>(c, 1);
    void* h = nullptr;
    check(c, cudaMallocHost(&h, 4 * sizeof(double) + sizeof(int)), "cudaMallocHost");
    c->hsc = static_cast<double*>(h);
    c->hflag = reinterpret_cast<int*>(c->hsc + 4);
    c->boxes = o.fused_transport != 0;
    // the box kernels may take more than the default 48 KB of shared memory
    const int maxb = (int)kBoxMaxBytes;
    check(c, cudaFuncSetAttribute(k3b_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb), "attr");
    check(c, cudaFuncSetAttribute(k3b_departure, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb), "attr");
    check(c, cudaFuncSetAttribute(k3b_adjoint_step, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb), "attr");
    check(c, cudaFuncSetAttribute(k3b_incstate_step, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb), "attr");
    if (two_level) {   // the coarse problem: same nt, model and options, P_REG inside
      reg_options oc = o;
      oc.precond = REG_PC_REG;
      const reg_status sc = reg3_create(n1 / 2, n2 / 2, n3 / 2, nt, beta, &oc, &c->coarse);
      if (sc != REG_OK) fail(c, sc, "coarse-grid context");
      const size_t Nc = (size_t)c->coarse->d.N;
      float** cvec[] = {&c->pc_rc, &c->pc_sc, &c->pc_r, &c->pc_d, &c->pc_w, &c->pc_u, &c->pc_q,
                        &c->pc_v};
      for (float** f : cvec) *f = dalloc<float>(c, 3 * Nc);
    }
    check(c, cudaDeviceSynchronize(), "create");
  });
  if (s != REG_OK) {
    reg3_destroy(c);
    return s;
  }
  *out = c;
  return REG_OK;
}

reg_status reg3_destroy(reg3_ctx* c) {
  if (!c) return REG_OK;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->coarse) reg3_destroy(c->coarse);
  for (void* p : c->allocs) cudaFree(p);
  if (c->hsc) cudaFreeHost(c->hsc);
  delete c;
  return REG_OK;
}

reg_status reg3_set_stream(reg3_ctx* c, void* stream) {
  if (!c) return REG_EINVAL;
  c->st = static_cast<cudaStream_t>(stream);
  if (c->coarse) c->coarse->st = c->st;
  return REG_OK;
}

reg_status reg3_set_images(reg3_ctx* c, const float* mR, const float* mT) {
  if (!c || !mR || !mT || unaligned(mR) || unaligned(mT)) return REG_EINVAL;
  return guarded(c, [&] {
    const size_t n = (size_t)c->d.N * sizeof(float);
    check(c, cudaMemcpyAsync(c->mR, mR, n, cudaMemcpyDeviceToDevice, c->st), "copy m_R");
    check(c, cudaMemcpyAsync(c->mT, mT, n, cudaMemcpyDeviceToDevice, c->st), "copy m_T");
    c->have_images = true;
    c->have_v = c->have_G = false;
    if (c->coarse) {
      restrict_images(c);
      c->have_eig = false;
    }
  });
}

reg_status reg3_transport(reg3_ctx* c, const float* v, const float* m0, float* m1) {
  if (!c || !v || !m0 || !m1 || unaligned(v) || unaligned(m0) || unaligned(m1)) return REG_EINVAL;
  return guarded(c, [&] {
    const long long N = c->d.N;
    if (v != c->v)
      check(c, cudaMemcpyAsync(c->v, v, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy v");
    departure(c, coefficients(c, c->v, 3, c->cv));
    check(c, cudaMemcpyAsync(c->fA, m0, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy m0");
    float* a = c->fA;
    float* b = c->fB;
    for (int j = 1; j <= c->nt; ++j) {
      gather(c, a, 1, c->dX, b, c->coef);
      std::swap(a, b);
    }
    check(c, cudaMemcpyAsync(m1, a, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy m1");
    c->have_v = false;   // the cached state no longer matches v
    c->have_G = false;
  });
}

// u = y - x of the deformation map of v (physical units, 3 fields) and, if
// det is not NULL, det grad y (§2, §4)
reg_status reg3_deformation_map(reg3_ctx* c, const float* v, float* u, float* det) {
  if (!c || !v || !u || unaligned(v) || unaligned(u) || (det && unaligned(det))) return REG_EINVAL;
  const long long N = c->d.N;
  if (det && det < u + 3 * N && u < det + N) return REG_EINVAL;   // overlapping outputs
  return guarded(c, [&] {
    if (v != c->v)
      check(c, cudaMemcpyAsync(c->v, v, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy v");
    departure(c, coefficients(c, c->v, 3, c->cv));
    const float h1 = (float)(2.0 * M_PI / c->d.n1), h2 = (float)(2.0 * M_PI / c->d.n2),
                h3 = (float)(2.0 * M_PI / c->d.n3);
    // u_0 = 0, u_j = u_{j-1}(X_D) + h dX (the first step without the gather of zeros)
    float* a = c->kx;
    float* nxt = c->kr;
    launch_fill(a, 3 * N, 0.f, c->st);
    launch_k(k3_add_disp, dim3(nb(N)), dim3(kT), 0, c->st, N, h1, h2, h3, (const float*)c->dX, a);
    for (int j = 2; j <= c->nt; ++j) {
      gather(c, a, 3, c->dX, nxt, c->c3);
      launch_k(k3_add_disp, dim3(nb(N)), dim3(kT), 0, c->st, N, h1, h2, h3, (const float*)c->dX, nxt);
      std::swap(a, nxt);
    }
    check(c, cudaMemcpyAsync(u, a, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy u");
    if (det) {
      grad_pair(c, a, c->gm);                                        // grad u_1, grad u_2
      spectral3(c, OP3_GRAD, 0.0, a + 2 * N, 1, c->b, 3, nullptr);   // grad u_3
      launch_k(k3_det_grad, dim3(nb(N)), dim3(kT), 0, c->st, N, (const float*)c->gm,
               (const float*)c->b, det);
    }
    check_launch(c, "deformation map");
    c->have_v = false;   // the characteristics and gradients of the cached velocity are gone
    c->have_G = false;
  });
}

reg_status reg3_spectral(reg3_ctx* c, int op, double s, const float* in, float* out) {
  if (!c || !in || !out || unaligned(in) || unaligned(out)) return REG_EINVAL;
  int fin, fout, o3;
  switch (op) {
    case REG_SPEC_GRAD: fin = 1; fout = 3; o3 = OP3_GRAD; break;
    case REG_SPEC_DIV: fin = 3; fout = 1; o3 = OP3_DIV; break;
    case REG_SPEC_REGPOW: fin = 3; fout = 3; o3 = OP3_REGPOW; break;
    default: return REG_EINVAL;
  }
  return guarded(c, [&] { spectral3(c, o3, s, in, fin, out, fout, nullptr); });
}

reg_status reg3_objective_gradient(reg3_ctx* c, const float* v, double* J, float* g) {
  if (!c || !v || !J || unaligned(v) || (g && unaligned(g))) return REG_EINVAL;
  return guarded(c, [&] {
    if (!c->have_images) fail(c, REG_ESTATE, "reg3_set_images has not been called");
    sync_velocity(c, v);
    *J = objective(c);
    if (g) gradient(c, g);
    check(c, cudaStreamSynchronize(c->st), "synchronize");
  });
}

reg_status reg3_hessian_matvec(reg3_ctx* c, const float* v, const float* vt, float* Hvt) {
  if (!c || !v || !vt || !Hvt || unaligned(v) || unaligned(vt) || unaligned(Hvt)) return REG_EINVAL;
  return guarded(c, [&] {
    if (!c->have_images) fail(c, REG_ESTATE, "reg3_set_images has not been called");
    sync_velocity(c, v);
    hessian(c, vt, Hvt);
    check(c, cudaStreamSynchronize(c->st), "synchronize");
  });
}

// The inexact Newton-Krylov solve of reg_solve (§3.4.1) on the 3D problem:
// ||g||_inf relative to g(0) as the stopping test, forcing term
// min(0.5, ||g|| / ||g(0)||), PCG with P_REG = (beta A)^-1, Armijo
// backtracking from the full step.
reg_status reg3_solve(reg3_ctx* c, float* v, double gtol, reg_info* info) {
  if (!c || !v || !(gtol > 0.0) || unaligned(v)) return REG_EINVAL;
  reg_info inf;
  std::memset(&inf, 0, sizeof inf);
  reg_status result = REG_OK;
  const auto t0 = std::chrono::steady_clock::now();
  const reg_status s = guarded(c, [&] {
    if (!c->have_images) fail(c, REG_ESTATE, "reg3_set_images has not been called");
    const reg_options& o = c->opt;
    const long long n = 3 * c->d.N;
    auto maxabs = [&](const float* a) {
      launch_maxabs(a, n, c->partialf, c->dsc, c->st);
      check(c, cudaMemcpyAsync(c->hsc, c->dsc, sizeof(double), cudaMemcpyDeviceToHost, c->st), "read");
      check(c, cudaStreamSynchronize(c->st), "synchronize");
      return c->hsc[0];
    };
    launch_fill(c->vtrial, n, 0.f, c->st);
    set_velocity(c, c->vtrial);
    objective(c);
    gradient(c, c->gcur);
    const double gref_inf = maxabs(c->gcur);
    const double gref_2 = std::sqrt(dot_sync(c, c->gcur, c->gcur, n));
    inf.gref_inf = gref_inf;
    const int cm0 = c->coarse_matvecs;
    const bool use_cheb = c->coarse && o.pc_solver == REG_PCSOLVER_CHEB;
    if (use_cheb && !c->have_eig) estimate_eig(c);
    set_velocity(c, v);
    double J = objective(c);
    inf.J0 = J;
    gradient(c, c->gcur);
    double rel = 1.0, ginf = 0.0;
    for (int k = 0;; ++k) {
      ginf = maxabs(c->gcur);
      if (!std::isfinite(ginf) || !std::isfinite(J)) { result = REG_ENONFINITE; break; }
      rel = ginf / gref_inf;
      if (rel <= gtol || ginf <= o.gabs) break;
      if (k == o.max_newton) { result = REG_ENOTCONV; break; }
      const double g2 = std::sqrt(dot_sync(c, c->gcur, c->gcur, n));
      const double eta = std::fmin(0.5, g2 / gref_2);
      c->eta = eta;
      if (c->coarse) set_velocity_coarse(c, v);
      // PCG (Hestenes-Stiefel) on H s = -g from s = 0 with P_REG
      launch_lincomb(n, -1.f, c->gcur, 0.f, nullptr, c->rhs, c->st);
      launch_fill(c->kx, n, 0.f, c->st);
      check(c, cudaMemcpyAsync(c->kr, c->rhs, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
      const double bnorm = std::sqrt(dot_sync(c, c->rhs, c->rhs, n));
      precond(c, c->kr, c->kz);
      check(c, cudaMemcpyAsync(c->kp, c->kz, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
      double rz = dot_sync(c, c->kr, c->kz, n);
      for (int it = 0; it < o.max_pcg && bnorm > 0.0; ++it) {
        hessian(c, c->kp, c->kq);
        ++inf.matvecs;
        const double pq = dot_sync(c, c->kp, c->kq, n);
        if (!(pq > 0.0)) {
          if (it == 0)
            check(c, cudaMemcpyAsync(c->kx, c->kz, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
          break;
        }
        const float alpha = (float)(rz / pq);
        launch_lincomb(n, 1.f, c->kx, alpha, c->kp, c->kx, c->st);
        launch_lincomb(n, 1.f, c->kr, -alpha, c->kq, c->kr, c->st);
        ++inf.pcg_iters;
        const double rr = dot_sync(c, c->kr, c->kr, n);
        if (std::sqrt(rr) / bnorm <= eta) break;
        precond(c, c->kr, c->kz);
        const double rz_new = dot_sync(c, c->kr, c->kz, n);
        launch_lincomb(n, 1.f, c->kz, (float)(rz_new / rz), c->kp, c->kp, c->st);
        rz = rz_new;
      }
      const double slope = c->hh * dot_sync(c, c->gcur, c->kx, n);
      double alpha = 1.0, Jt = J;
      bool ok = false;
      for (int ls = 0; ls <= o.max_backtracks; ++ls) {
        launch_lincomb(n, 1.f, v, (float)alpha, c->kx, c->vtrial, c->st);
        set_velocity(c, c->vtrial);
        Jt = objective(c);
        ++inf.line_search_steps;
        if (Jt <= J + o.armijo_c1 * alpha * slope) { ok = true; break; }
        alpha *= 0.5;
      }
      if (!ok) {
        set_velocity(c, v);
        objective(c);
        result = REG_ELINESEARCH;
        break;
      }
      check(c, cudaMemcpyAsync(v, c->vtrial, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "accept");
      J = Jt;
      gradient(c, c->gcur);
      ++inf.newton_iters;
    }
    inf.J = J;
    inf.gnorm_rel = rel;
    inf.gnorm_inf = ginf;
    inf.coarse_matvecs = c->coarse_matvecs - cm0;
    check(c, cudaStreamSynchronize(c->st), "synchronize");
  });
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (s != REG_OK) result = s;
  inf.status = result;
  if (info) *info = inf;
  return result;
}

reg_status reg3_precond_apply(reg3_ctx* c, const float* v, const float* r, float* z) {
  if (!c || !v || !r || !z || r == z || unaligned(v) || unaligned(r) || unaligned(z)) return REG_EINVAL;
  return guarded(c, [&] {
    if (c->coarse) {
      if (!c->have_images) fail(c, REG_ESTATE, "reg3_set_images has not been called");
      if (c->opt.pc_solver == REG_PCSOLVER_CHEB && !c->have_eig) estimate_eig(c);
      set_velocity_coarse(c, v);
    }
    precond(c, r, z);
    check(c, cudaStreamSynchronize(c->st), "synchronize");
  });
}

reg_status reg3_eigen_bounds(reg3_ctx* c, double* emin, double* emax) {
  if (!c || !emin || !emax) return REG_EINVAL;
  return guarded(c, [&] {
    if (!c->coarse) fail(c, REG_EINVAL, "the context runs P_REG");
    if (!c->have_images) fail(c, REG_ESTATE, "reg3_set_images has not been called");
    estimate_eig(c);
    check(c, cudaStreamSynchronize(c->st), "synchronize");
    *emin = c->emin;
    *emax = c->emax;
  });
}

const char* reg3_last_error(const reg3_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
