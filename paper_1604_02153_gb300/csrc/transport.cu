// Semi-Lagrangian kernels: spline prefilter, RK2 departure points, periodic
// 4x4 cubic interpolation and the fused transport steps of the state,
// adjoint, incremental state and incremental adjoint equations
// (§3.3.2, eq. hyperbolic-pdes-slm, eq. characteristic,
// eq. transport-along-characteristic; §3.5 "Interpolation").
//
// Displacements are stored in cell units, d = (X_D - x) / h, so that the
// node index and the sub-cell offset stay separate in FP32: the stencil base
// is i + floor(d) and the weights use t = d - floor(d), both exact.
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "interp.cuh"
#include "kernels.h"

namespace regnk {

// True when both grid lengths are powers of two (see split_index).
static bool pow2_grid(int n1, int n2) { return !(n1 & (n1 - 1)) && !(n2 & (n2 - 1)); }

// log2(n) for powers of two, -1 otherwise
static int ilog2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return (1 << l) == n ? l : -1;
}

// The instantiation of a kernel template for the grid's index arithmetic.
template <typename K>
static K pick(int n1, int n2, K p2, K general) { return pow2_grid(n1, n2) ? p2 : general; }

// One block per 32x32 output tile and field.
template <bool P2>
__global__ void __launch_bounds__(kPThreads)
k_prefilter(const float* __restrict__ in, float* __restrict__ out, int n1, int n2, int log1,
            long long fstride) {
  pdl_enter();
  __shared__ float sin_[kPH * kPIn];
  __shared__ float smid[kPH * kPMid];
  const long long fo = (long long)blockIdx.z * fstride;
  prefilter_tile<P2>(in + fo, out + fo, n1, n2, log1, blockIdx.x * kPX, blockIdx.y * kPY, sin_,
                     smid);
}

void launch_prefilter(int n1, int n2, const float* in, float* tmp, float* out, int F,
                      cudaStream_t st) {
  (void)tmp;
  launch_k(pick(n1, n2, k_prefilter<true>, k_prefilter<false>), dim3(n1 / kPX, n2 / kPY, F),
           dim3(kPThreads), 0, st, in, out, n1, n2, ilog2i(n1), (long long)n1 * n2);
}

constexpr int kPT = 256;  // threads per block of the pointwise kernels

// Departure points of both characteristics (Heun, §3.3.2):
//   X* = x - h_t v(x),  X_D = x - h_t/2 (v(x) + v(X*))
//   Y* = x + h_t v(x),  Y_D = x + h_t/2 (v(x) + v(Y*))
// cv holds the interpolation coefficients of v (spline) or v itself.
template <bool P2>
__device__ __forceinline__ void departure_point(long long idx, int n1, int n2, int log1, float s1,
                                                float s2, const float* __restrict__ v,
                                                const float* __restrict__ cv,
                                                float* __restrict__ dX, float* __restrict__ dY,
                                                int lagrange) {
  const long long N = (long long)n1 * n2;
  int i, j;
  split_index<P2>(idx, n1, log1, i, j);
  const float v1 = __ldg(v + idx), v2 = __ldg(v + N + idx);
  const float a1 = s1 * v1, a2 = s2 * v2;   // h_t v / h in cells
  if (dX) {
    const Stencil S = make_stencil<P2>(i, j, -a1, -a2, n1, n2, log1, lagrange);
    const float w1 = apply_stencil(S, cv), w2 = apply_stencil(S, cv + N);
    dX[idx] = -0.5f * (a1 + s1 * w1);
    dX[N + idx] = -0.5f * (a2 + s2 * w2);
  }
  if (dY) {
    const Stencil S = make_stencil<P2>(i, j, a1, a2, n1, n2, log1, lagrange);
    const float w1 = apply_stencil(S, cv), w2 = apply_stencil(S, cv + N);
    dY[idx] = 0.5f * (a1 + s1 * w1);
    dY[N + idx] = 0.5f * (a2 + s2 * w2);
  }
}

template <bool P2>
__global__ void __launch_bounds__(kPT)
k_departure(int n1, int n2, int log1, float s1, float s2, const float* __restrict__ v,
            const float* __restrict__ cv, float* __restrict__ dX, float* __restrict__ dY,
            int lagrange) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= (long long)n1 * n2) return;
  departure_point<P2>(idx, n1, n2, log1, s1, s2, v, cv, dX, dY, lagrange);
}

float departure_scale(float ht, int n) { return ht * n / (2.0f * 3.14159265358979323846f); }

void launch_departure(int n1, int n2, float ht, const float* v, const float* cv, float* dX,
                      float* dY, int lagrange, cudaStream_t st) {
  const long long N = (long long)n1 * n2;
  const float s1 = departure_scale(ht, n1);
  const float s2 = departure_scale(ht, n2);
  launch_k(pick(n1, n2, k_departure<true>, k_departure<false>), dim3((unsigned)((N + kPT - 1) / kPT)),
           dim3(kPT), 0, st, n1, n2, ilog2i(n1), s1, s2, v, cv, dX, dY, lagrange);
}

// The step kernels below (k_adjoint_step, k_incstate_step) handle SP
// horizontally adjacent points per thread in blocks of T threads (row lengths
// are multiples of 32, so the SP points of a thread share a row): their
// streamed fields move as SP-float vectors and the SP independent 4x4
// stencils keep more loads in flight per thread. (SP, T) is the tile shape,
// chosen per grid level at run time among kStepTiles shapes (index k = 1..9:
// T = 128 << ((k - 1) / 3), SP = 1 << ((k - 1) % 3)). Every point's
// arithmetic is the same in every shape.
#define REGNK_STEP_TILES(X) \
  X(1, 1, 128) X(2, 2, 128) X(3, 4, 128) X(4, 1, 256) X(5, 2, 256) X(6, 4, 256) \
  X(7, 1, 512) X(8, 2, 512) X(9, 4, 512)

template <int K>
__device__ __forceinline__ void ldk(const float* p, float (&a)[K]) {
  if constexpr (K == 1) {
    a[0] = __ldg(p);
  } else if constexpr (K == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    a[0] = t.x; a[1] = t.y;
  } else {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
  }
}

// plain (not read-only) load, for buffers the kernel also writes
template <int K>
__device__ __forceinline__ void ldk_rw(const float* p, float (&a)[K]) {
  if constexpr (K == 1) {
    a[0] = *p;
  } else if constexpr (K == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    a[0] = t.x; a[1] = t.y;
  } else {
    const float4 t = *reinterpret_cast<const float4*>(p);
    a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
  }
}

template <int K>
__device__ __forceinline__ void stk(float* p, const float (&a)[K]) {
  if constexpr (K == 1) {
    *p = a[0];
  } else if constexpr (K == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(a[0], a[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(a[0], a[1], a[2], a[3]);
  }
}

template <int SP, int T>
static unsigned step_blocks(long long N) { return (unsigned)((N / SP + T - 1) / T); }

// out_f = I[coef_f](x + disp), f = 0..F-1 (fields fstride apart), one stencil
// per point, one point per thread; F = 1 or 2 is a compile-time constant so
// that the loads of both fields are in flight together without the
// register cost of an unrolled loop of unknown length.
template <bool P2, int F>
__global__ void __launch_bounds__(kPT)
k_gather(int n1, int n2, int log1, const float* __restrict__ coef,
         const float* __restrict__ disp, float* __restrict__ out, long long fstride,
         int lagrange) {
  pdl_enter();
  const long long N = (long long)n1 * n2;
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  int i, j;
  split_index<P2>(idx, n1, log1, i, j);
  const Stencil S = make_stencil<P2>(i, j, __ldg(disp + idx), __ldg(disp + N + idx), n1, n2,
                                     log1, lagrange);
  float o[F];
#pragma unroll
  for (int f = 0; f < F; ++f) o[f] = apply_stencil(S, coef + f * fstride);
#pragma unroll
  for (int f = 0; f < F; ++f) out[f * fstride + idx] = o[f];
}

template <int F>
static void gather_f(int n1, int n2, const float* coef, const float* disp, float* out,
                     long long fstride, int lagrange, cudaStream_t st) {
  const long long N = (long long)n1 * n2;
  const unsigned nb = (unsigned)((N + kPT - 1) / kPT);
  launch_k(pick(n1, n2, k_gather<true, F>, k_gather<false, F>), dim3(nb), dim3(kPT), 0, st, n1, n2,
           ilog2i(n1), coef, disp, out, fstride, lagrange);
}

void launch_gather(int n1, int n2, const float* coef, const float* disp, float* out, int F,
                   long long fstride, int lagrange, cudaStream_t st) {
  // callers interpolate one scalar field or one vector field
  if (F == 2)
    gather_f<2>(n1, n2, coef, disp, out, fstride, lagrange, st);
  else
    gather_f<1>(n1, n2, coef, disp, out, fstride, lagrange, st);
}

void launch_state_step(int n1, int n2, const float* coef, const float* dX, float* out,
                       int lagrange, cudaStream_t st) {
  launch_gather(n1, n2, coef, dX, out, 1, 0, lagrange, st);
}

// Final condition of an adjoint solve and the first term of its time
// integral: lam = sign * (mR - m1) (mR may be NULL: lam = -sign * m1),
// b = coef_b * lam * grad m.
__device__ __forceinline__ void adjoint_init_point(long long idx, long long N, float coef_b,
                                                   const float* __restrict__ mR,
                                                   const float* __restrict__ m1,
                                                   const float* __restrict__ gm,
                                                   float* __restrict__ lam, float* __restrict__ b,
                                                   float sign) {
  const float r = (mR ? __ldg(mR + idx) : 0.f) - __ldg(m1 + idx);
  const float l = sign * r;
  lam[idx] = l;
  b[idx] = coef_b * l * __ldg(gm + idx);
  b[N + idx] = coef_b * l * __ldg(gm + N + idx);
}

__global__ void __launch_bounds__(kPT)
k_adjoint_init(long long N, float coef_b, const float* __restrict__ mR,
               const float* __restrict__ m1, const float* __restrict__ gm,
               float* __restrict__ lam, float* __restrict__ b, float sign) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  adjoint_init_point(idx, N, coef_b, mR, m1, gm, lam, b, sign);
}

void launch_adjoint_init(int n1, int n2, float coef_b, const float* mR, const float* m1,
                         const float* gm, float* lam, float* b, float sign, cudaStream_t st) {
  const long long N = (long long)n1 * n2;
  launch_k(k_adjoint_init, dim3((unsigned)((N + kPT - 1) / kPT)), dim3(kPT), 0, st, N, coef_b, mR,
           m1, gm, lam, b, sign);
}

// One backward step of the (incremental) adjoint along Y_D (§3.3.2, Heun):
//   lb = lam_{j+1}(Y_D), lam* = lb + h_t lb div v(Y_D),
//   lam_j = lb + h_t/2 (lb div v(Y_D) + lam* div v(x)),
// fused with the time integral b += wb * lam_j * grad m_j.
template <bool P2, int SP, int T>
__global__ void __launch_bounds__(T)
k_adjoint_step(int n1, int n2, int log1, float ht, float wb, const float* __restrict__ coef,
               const float* __restrict__ dY, const float* __restrict__ delta,
               const float* __restrict__ delta_bar, const float* __restrict__ gm,
               float* __restrict__ lam_out, float* __restrict__ b, int lagrange) {
  pdl_enter();
  const long long N = (long long)n1 * n2;
  const long long idx = SP * ((long long)blockIdx.x * T + threadIdx.x);
  if (idx >= N) return;
  int i, j;
  split_index<P2>(idx, n1, log1, i, j);
  // every streamed operand is requested together with the displacement, so
  // that their latency overlaps the dependent gather
  float y1[SP], y2[SP], l[SP], db[SP], d[SP], g1[SP], g2[SP], b1[SP], b2[SP];
  ldk(dY + idx, y1);
  ldk(dY + N + idx, y2);
  ldk(delta_bar + idx, db);
  ldk(delta + idx, d);
  ldk(gm + idx, g1);
  ldk(gm + N + idx, g2);
  ldk_rw(b + idx, b1);
  ldk_rw(b + N + idx, b2);
#pragma unroll
  for (int p = 0; p < SP; ++p)
    l[p] = apply_stencil(make_stencil<P2>(i + p, j, y1[p], y2[p], n1, n2, log1, lagrange), coef);
#pragma unroll
  for (int p = 0; p < SP; ++p) {
    const float lstar = fmaf(ht * l[p], db[p], l[p]);
    l[p] = l[p] + 0.5f * ht * (l[p] * db[p] + lstar * d[p]);
  }
  stk(lam_out + idx, l);
#pragma unroll
  for (int p = 0; p < SP; ++p) {
    b1[p] = fmaf(wb * l[p], g1[p], b1[p]);
    b2[p] = fmaf(wb * l[p], g2[p], b2[p]);
  }
  stk(b + idx, b1);
  stk(b + N + idx, b2);
}

template <int SP, int T>
static void adjoint_step_t(int n1, int n2, float ht, float wb, const float* coef, const float* dY,
                           const float* delta, const float* delta_bar, const float* gm,
                           float* lam_out, float* b, int lagrange, cudaStream_t st) {
  const long long N = (long long)n1 * n2;
  launch_k(pick(n1, n2, k_adjoint_step<true, SP, T>, k_adjoint_step<false, SP, T>),
           dim3(step_blocks<SP, T>(N)), dim3(T), 0, st, n1, n2, ilog2i(n1), ht, wb, coef, dY, delta,
           delta_bar, gm, lam_out, b, lagrange);
}

void launch_adjoint_step(int tile, int n1, int n2, float ht, float wb, const float* coef,
                         const float* dY, const float* delta, const float* delta_bar,
                         const float* gm, float* lam_out, float* b, int lagrange,
                         cudaStream_t st) {
  switch (tile) {
#define REGNK_ADJ_CASE(K, SP, T) \
  case K: adjoint_step_t<SP, T>(n1, n2, ht, wb, coef, dY, delta, delta_bar, gm, lam_out, b, lagrange, st); break;
    REGNK_STEP_TILES(REGNK_ADJ_CASE)
#undef REGNK_ADJ_CASE
    default: adjoint_step_t<2, 256>(n1, n2, ht, wb, coef, dY, delta, delta_bar, gm, lam_out, b, lagrange, st);
  }
}

// One forward step of the incremental state (Gauss-Newton, §3.3.2):
//   m~_j = m~_{j-1}(X_D) - h_t/2 (v~(X_D) . grad m_{j-1}(X_D) + v~ . grad m_j)
// G = grad m_{j-1}(X_D) (2 fields), vtD = v~(X_D) (2 fields), gm = grad m_j.
// first = 1 for j = 1 where m~_0 = 0; then, if cvt (the interpolation
// coefficients of v~, or v~ itself for the Lagrange model) is given, v~(X_D)
// is gathered here and written to vtD instead of being read from it.
// gm_nt, b: non-NULL for the last step j = nt, which writes
// lambda~_nt = -m~_nt and b = h_t/2 lambda~_nt grad m_nt (k_adjoint_init).
template <bool P2, int SP, int T>
__global__ void __launch_bounds__(T)
k_incstate_step(int n1, int n2, int log1, float ht, const float* __restrict__ coef,
                const float* __restrict__ dX, const float* __restrict__ vt,
                float* __restrict__ vtD, const float* __restrict__ G,
                const float* __restrict__ gm, float* __restrict__ out, int first,
                int lagrange, const float* __restrict__ cvt, const float* __restrict__ gm_nt,
                float* __restrict__ b) {
  pdl_enter();
  const long long N = (long long)n1 * n2;
  const long long idx = SP * ((long long)blockIdx.x * T + threadIdx.x);
  if (idx >= N) return;
  float m[SP], w1[SP], w2[SP];
#pragma unroll
  for (int p = 0; p < SP; ++p) m[p] = 0.f;
  // the streamed operands are requested before the dependent gather
  float G1[SP], G2[SP], u1[SP], u2[SP], g1[SP], g2[SP];
  ldk(G + idx, G1);
  ldk(G + N + idx, G2);
  ldk(vt + idx, u1);
  ldk(vt + N + idx, u2);
  ldk(gm + idx, g1);
  ldk(gm + N + idx, g2);
  if (!cvt) {
    ldk(vtD + idx, w1);
    ldk(vtD + N + idx, w2);
  }
  float gn1[SP], gn2[SP];
  if (b) {
    ldk(gm_nt + idx, gn1);
    ldk(gm_nt + N + idx, gn2);
  }
  if (!first || cvt) {
    int i, j;
    split_index<P2>(idx, n1, log1, i, j);
    float x1[SP], x2[SP];
    ldk(dX + idx, x1);
    ldk(dX + N + idx, x2);
#pragma unroll
    for (int p = 0; p < SP; ++p) {
      const Stencil S = make_stencil<P2>(i + p, j, x1[p], x2[p], n1, n2, log1, lagrange);
      if (!first) m[p] = apply_stencil(S, coef);
      if (cvt) {
        w1[p] = apply_stencil(S, cvt);
        w2[p] = apply_stencil(S, cvt + N);
      }
    }
  }
  if (cvt) {
    stk(vtD + idx, w1);
    stk(vtD + N + idx, w2);
  }
#pragma unroll
  for (int p = 0; p < SP; ++p)
    m[p] -= 0.5f * ht * (w1[p] * G1[p] + w2[p] * G2[p] + u1[p] * g1[p] + u2[p] * g2[p]);
  if (!b) {
    stk(out + idx, m);
    return;
  }
  float lam[SP], b1[SP], b2[SP];
  const float hh = 0.5f * ht;
#pragma unroll
  for (int p = 0; p < SP; ++p) {
    lam[p] = -m[p];
    b1[p] = hh * lam[p] * gn1[p];
    b2[p] = hh * lam[p] * gn2[p];
  }
  stk(out + idx, lam);
  stk(b + idx, b1);
  stk(b + N + idx, b2);
}

template <int SP, int T>
static void incstate_step_t(int n1, int n2, float ht, const float* coef, const float* dX,
                            const float* vt, float* vtD, const float* G, const float* gm,
                            float* out, int first, int lagrange, cudaStream_t st,
                            const float* cvt, const float* gm_nt, float* b) {
  const long long N = (long long)n1 * n2;
  launch_k(pick(n1, n2, k_incstate_step<true, SP, T>, k_incstate_step<false, SP, T>),
           dim3(step_blocks<SP, T>(N)), dim3(T), 0, st, n1, n2, ilog2i(n1), ht, coef, dX, vt, vtD,
           G, gm, out, first, lagrange, cvt, gm_nt, b);
}

void launch_incstate_step(int tile, int n1, int n2, float ht, const float* coef, const float* dX,
                          const float* vt, float* vtD, const float* G, const float* gm,
                          float* out, int first, int lagrange, cudaStream_t st,
                          const float* cvt, const float* gm_nt, float* b) {
  switch (tile) {
#define REGNK_INC_CASE(K, SP, T)                                                                 \
  case K:                                                                                        \
    incstate_step_t<SP, T>(n1, n2, ht, coef, dX, vt, vtD, G, gm, out, first, lagrange, st, cvt,  \
                           gm_nt, b);                                                            \
    break;
    REGNK_STEP_TILES(REGNK_INC_CASE)
#undef REGNK_INC_CASE
    default:
      incstate_step_t<2, 256>(n1, n2, ht, coef, dX, vt, vtD, G, gm, out, first, lagrange, st, cvt,
                              gm_nt, b);
  }
}

// ---------------------------------------------------------------------------
// Full-Newton incremental adjoint (eq. inc-adj-slm with the div(lambda v~)
// source) and the time integral of lambda~ grad m + lambda grad m~
// (eq. hessian-matvec as written). One point per thread.

// out[j][c] = lam_j * vt_c, j = 0..L-1, c = 0, 1 (the fields whose divergence
// is the source of the full-Newton incremental adjoint)
__global__ void __launch_bounds__(kPT)
k_lam_times_vt(long long N, int L, const float* __restrict__ lam, const float* __restrict__ vt,
               float* __restrict__ out) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N * L) return;
  const long long j = idx / N, i = idx - j * N;
  const float l = __ldg(lam + idx);
  out[2 * j * N + i] = l * __ldg(vt + i);
  out[(2 * j + 1) * N + i] = l * __ldg(vt + N + i);
}

void launch_lam_times_vt(long long N, int L, const float* lam, const float* vt, float* out,
                         cudaStream_t st) {
  launch_k(k_lam_times_vt, dim3((unsigned)((N * L + kPT - 1) / kPT)), dim3(kPT), 0, st, N, L, lam,
           vt, out);
}

// lam~_nt = -m~_nt; b~ = coef_b (lam~_nt grad m_nt + lam_nt grad m~_nt)
__global__ void __launch_bounds__(kPT)
k_fn_adjoint_init(long long N, float coef_b, const float* __restrict__ mt,
                  const float* __restrict__ gm, const float* __restrict__ lam,
                  const float* __restrict__ gmt, float* __restrict__ lt, float* __restrict__ b) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  const float l = -__ldg(mt + idx);
  const float a = __ldg(lam + idx);
  lt[idx] = l;
  b[idx] = coef_b * (l * __ldg(gm + idx) + a * __ldg(gmt + idx));
  b[N + idx] = coef_b * (l * __ldg(gm + N + idx) + a * __ldg(gmt + N + idx));
}

void launch_fn_adjoint_init(long long N, float coef_b, const float* mt, const float* gm,
                            const float* lam, const float* gmt, float* lt, float* b,
                            cudaStream_t st) {
  launch_k(k_fn_adjoint_init, dim3((unsigned)((N + kPT - 1) / kPT)), dim3(kPT), 0, st, N, coef_b,
           mt, gm, lam, gmt, lt, b);
}

// One backward step (Heun, reversed time): with lb = lam~_{j+1}(Y_D) and
// sb = s_{j+1}(Y_D), s_j = div(lambda_j v~),
//   f = lb div v(Y_D) + sb,  lam* = lb + h_t f,
//   lam~_j = lb + h_t/2 (f + lam* div v + s_j),
// then b~ += wb (lam~_j grad m_j + lambda_j grad m~_j) (gmt NULL: grad m~_0 = 0).
// coef_l, coef_s: interpolation coefficients of lam~_{j+1} and s_{j+1}.
template <bool P2>
__global__ void __launch_bounds__(kPT)
k_fn_adjoint_step(int n1, int n2, int log1, float ht, float wb, const float* __restrict__ coef_l,
                  const float* __restrict__ coef_s, const float* __restrict__ dY,
                  const float* __restrict__ delta, const float* __restrict__ delta_bar,
                  const float* __restrict__ src, const float* __restrict__ gm,
                  const float* __restrict__ lam, const float* __restrict__ gmt,
                  float* __restrict__ lt_out, float* __restrict__ b, int lagrange) {
  pdl_enter();
  const long long N = (long long)n1 * n2;
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  int i, j;
  split_index<P2>(idx, n1, log1, i, j);
  const Stencil S = make_stencil<P2>(i, j, __ldg(dY + idx), __ldg(dY + N + idx), n1, n2, log1,
                                     lagrange);
  const float lb = apply_stencil(S, coef_l);
  const float sb = apply_stencil(S, coef_s);
  const float f = fmaf(lb, __ldg(delta_bar + idx), sb);
  const float lstar = fmaf(ht, f, lb);
  const float l = lb + 0.5f * ht * (f + fmaf(lstar, __ldg(delta + idx), __ldg(src + idx)));
  lt_out[idx] = l;
  const float a = __ldg(lam + idx);
  const float t1 = gmt ? a * __ldg(gmt + idx) : 0.f;
  const float t2 = gmt ? a * __ldg(gmt + N + idx) : 0.f;
  b[idx] = fmaf(wb, fmaf(l, __ldg(gm + idx), t1), b[idx]);
  b[N + idx] = fmaf(wb, fmaf(l, __ldg(gm + N + idx), t2), b[N + idx]);
}

void launch_fn_adjoint_step(int n1, int n2, float ht, float wb, const float* coef_l,
                            const float* coef_s, const float* dY, const float* delta,
                            const float* delta_bar, const float* src, const float* gm,
                            const float* lam, const float* gmt, float* lt_out, float* b,
                            int lagrange, cudaStream_t st) {
  const long long N = (long long)n1 * n2;
  launch_k(pick(n1, n2, k_fn_adjoint_step<true>, k_fn_adjoint_step<false>),
           dim3((unsigned)((N + kPT - 1) / kPT)), dim3(kPT), 0, st, n1, n2, ilog2i(n1), ht, wb,
           coef_l, coef_s, dY, delta, delta_bar, src, gm, lam, gmt, lt_out, b, lagrange);
}

// ---------------------------------------------------------------------------
// RK2A comparator (antisymmetric form, Appendix "RK2A derivation"): one Heun
// stage. With g = grad u, dv = div(u v) (spectral) and delta = div v,
//   k = 1/2 (s (g . v + dv) + u delta),
// s = -1 for the state equation, +1 for the adjoint in reversed time; then
// out = base + a k (+ b kprev) and, if kout, kout = k. out may be base.
__global__ void __launch_bounds__(kPT)
k_rk2a_stage(long long N, float s, const float* __restrict__ u, const float* __restrict__ g,
             const float* __restrict__ v, const float* __restrict__ dv,
             const float* __restrict__ delta, const float* base, float a,
             const float* __restrict__ kprev, float b, float* out, float* __restrict__ kout) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  const float adv = fmaf(__ldg(g + idx), __ldg(v + idx), fmaf(__ldg(g + N + idx), __ldg(v + N + idx),
                                                               __ldg(dv + idx)));
  const float k = 0.5f * fmaf(s, adv, __ldg(u + idx) * __ldg(delta + idx));
  if (kout) kout[idx] = k;
  float o = fmaf(a, k, base[idx]);
  if (kprev) o = fmaf(b, __ldg(kprev + idx), o);
  out[idx] = o;
}

void launch_rk2a_stage(long long N, float s, const float* u, const float* g, const float* v,
                       const float* dv, const float* delta, const float* base, float a,
                       const float* kprev, float b, float* out, float* kout, cudaStream_t st) {
  launch_k(k_rk2a_stage, dim3((unsigned)((N + kPT - 1) / kPT)), dim3(kPT), 0, st, N, s, u, g, v, dv,
           delta, base, a, kprev, b, out, kout);
}

// det grad y for y = x + u from the spectral derivatives g = [d1 u1, d2 u1,
// d1 u2, d2 u2] (4 fields): (1 + d1 u1)(1 + d2 u2) - d2 u1 d1 u2.
__global__ void __launch_bounds__(kPT)
k_det_grad(long long N, const float* __restrict__ g, float* __restrict__ det) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  const float a = 1.f + __ldg(g + idx), b = __ldg(g + N + idx);
  const float c = __ldg(g + 2 * N + idx), d = 1.f + __ldg(g + 3 * N + idx);
  det[idx] = fmaf(a, d, -b * c);
}

void launch_det_grad(long long N, const float* g, float* det, cudaStream_t st) {
  launch_k(k_det_grad, dim3((unsigned)((N + kPT - 1) / kPT)), dim3(kPT), 0, st, N, g, det);
}

// ---------------------------------------------------------------------------
// Fused steps: the spline prefilter of the field being transported and the
// step that gathers it, in one kernel. A block owns a 32x32 tile of output
// points. Every stencil of the tile lies in the W x W box of nodes that
// extends the tile by H = (W - 32) / 2 on each side when all displacements
// satisfy |d| <= H - 2 cells (the host checks the velocity's largest
// displacement before choosing this path). The block computes the spline
// coefficients of that box from the raw samples (prefilter_box, with the
// same recursion segments as k_prefilter since H is a multiple of 8, so the
// coefficients and the results are bitwise those of the two-kernel path)
// and gathers from shared memory. Each thread handles kFP points of a tile
// row, kFS apart.

template <int W>
__device__ __forceinline__ void box_stencil(int lx, int ly, float d1, float d2, bool lagrange,
                                            int& li, int& lj, float (&w1)[4], float (&w2)[4]) {
  const float f1 = floorf(d1), f2 = floorf(d2);
  cubic_weights(d1 - f1, w1, lagrange);
  cubic_weights(d2 - f2, w2, lagrange);
  li = min(max(lx + (int)f1 - 1, 0), W - 4);
  lj = min(max(ly + (int)f2 - 1, 0), W - 4);
}

// threads of the fused kernels: one round of recursions per pass for the
// 48^2 box (74 x 6 x-segments, 48 x 6 y-segments) and two points per thread
constexpr int kFT = 512;
constexpr int kFP = 1024 / kFT;   // points per thread
constexpr int kFS = 32 / kFP;     // their spacing along the tile row

// The kFP points of a thread in a fused kernel are kFS apart in the tile row,
// so that the 16 lanes of a warp on one tile row touch consecutive columns for
// each point (adjacent points per thread gave 2-way conflicts) and the
// streamed loads and stores stay coalesced; with the box pitch 16 mod 32 the
// warp's two tile rows fall in opposite halves of the banks, so a 4x4 gather
// conflicts only where the stencil bases of neighbouring points jump.
template <int K>
__device__ __forceinline__ void ldf(const float* p, float (&a)[K]) {
#pragma unroll
  for (int q = 0; q < K; ++q) a[q] = __ldg(p + q * kFS);
}

template <int K>
__device__ __forceinline__ void ldf_rw(const float* p, float (&a)[K]) {
#pragma unroll
  for (int q = 0; q < K; ++q) a[q] = p[q * kFS];
}

template <int K>
__device__ __forceinline__ void stf(float* p, const float (&a)[K]) {
#pragma unroll
  for (int q = 0; q < K; ++q) p[q * kFS] = a[q];
}

// The bodies of the fused kernels take the tile origin (x0, y0) and the
// block's dynamic shared memory, so that the one-problem kernels (tile =
// blockIdx) and the batched kernels (tile from a table over many problems)
// run the same code.
template <bool P2, int W>
__device__ __forceinline__ void adjoint_fused_body(
    int n1, int n2, int log1, int x0, int y0, float* sm, float ht, float wb,
    const float* __restrict__ lam_next, const float* __restrict__ dY,
    const float* __restrict__ delta, const float* __restrict__ delta_bar,
    const float* __restrict__ gm, float* __restrict__ lam_out, float* __restrict__ b) {
  using D = BoxDims<W>;
  constexpr int H = (W - 32) / 2;
  float* stage = sm;
  float* mid = sm + D::kStage;
  const long long N = (long long)n1 * n2;
  constexpr int TPR = 32 / kFP;   // threads per tile row
  const int t = threadIdx.x, r = t / TPR, cx = t % TPR;
  const long long idx = row_offset<P2>(y0 + r, n1, log1) + x0 + cx;
  // the step's streamed operands are loaded first: their latency overlaps
  // the staging and the recursions of the prefilter
  float y1[kFP], y2[kFP], db[kFP], dd[kFP], g1[kFP], g2[kFP], b1[kFP], b2[kFP];
  ldf(dY + idx, y1);
  ldf(dY + N + idx, y2);
  ldf(delta_bar + idx, db);
  ldf(delta + idx, dd);
  ldf(gm + idx, g1);
  ldf(gm + N + idx, g2);
  ldf_rw(b + idx, b1);
  ldf_rw(b + N + idx, b2);
  prefilter_box<W, P2, kFT>(lam_next, n1, n2, log1, x0 - H, y0 - H, stage, mid, stage);
  float l[kFP];
#pragma unroll
  for (int p = 0; p < kFP; ++p) {
    int li, lj;
    float w1[4], w2[4];
    box_stencil<W>(H + cx + kFS * p, H + r, y1[p], y2[p], false, li, lj, w1, w2);
    const float lb = apply_box<D::PB>(stage, li, lj, w1, w2);
    const float lstar = fmaf(ht * lb, db[p], lb);
    l[p] = lb + 0.5f * ht * (lb * db[p] + lstar * dd[p]);
    b1[p] = fmaf(wb * l[p], g1[p], b1[p]);
    b2[p] = fmaf(wb * l[p], g2[p], b2[p]);
  }
  stf(lam_out + idx, l);
  stf(b + idx, b1);
  stf(b + N + idx, b2);
}

template <bool P2, int W>
__global__ void __launch_bounds__(kFT, 2)
k_adjoint_fused(int n1, int n2, int log1, float ht, float wb, const float* __restrict__ lam_next,
                const float* __restrict__ dY, const float* __restrict__ delta,
                const float* __restrict__ delta_bar, const float* __restrict__ gm,
                float* __restrict__ lam_out, float* __restrict__ b) {
  pdl_enter();
  extern __shared__ float sm[];
  adjoint_fused_body<P2, W>(n1, n2, log1, blockIdx.x * 32, blockIdx.y * 32, sm, ht, wb, lam_next,
                            dY, delta, delta_bar, gm, lam_out, b);
}

// gm_nt, b: non-NULL for the last step j = nt, which writes the final
// condition of the incremental adjoint, lambda~_nt = -m~_nt, to `out` and
// starts its time integral, b = h_t/2 lambda~_nt grad m_nt (the work of
// k_adjoint_init).
template <bool P2, int W>
__device__ __forceinline__ void incstate_fused_body(
    int n1, int n2, int log1, int x0, int y0, float* sm, float ht,
    const float* __restrict__ m_prev, const float* __restrict__ dX, const float* __restrict__ vt,
    const float* __restrict__ vtD, const float* __restrict__ G, const float* __restrict__ gm,
    float* __restrict__ out, const float* __restrict__ gm_nt, float* __restrict__ b) {
  using D = BoxDims<W>;
  constexpr int H = (W - 32) / 2;
  float* stage = sm;
  float* mid = sm + D::kStage;
  const long long N = (long long)n1 * n2;
  constexpr int TPR = 32 / kFP;
  const int t = threadIdx.x, r = t / TPR, cx = t % TPR;
  const long long idx = row_offset<P2>(y0 + r, n1, log1) + x0 + cx;
  // streamed operands first (their latency overlaps the prefilter)
  float x1[kFP], x2[kFP], w1v[kFP], w2v[kFP], G1[kFP], G2[kFP], u1[kFP], u2[kFP], g1[kFP], g2[kFP];
  ldf(dX + idx, x1);
  ldf(dX + N + idx, x2);
  ldf(vtD + idx, w1v);
  ldf(vtD + N + idx, w2v);
  ldf(G + idx, G1);
  ldf(G + N + idx, G2);
  ldf(vt + idx, u1);
  ldf(vt + N + idx, u2);
  ldf(gm + idx, g1);
  ldf(gm + N + idx, g2);
  prefilter_box<W, P2, kFT>(m_prev, n1, n2, log1, x0 - H, y0 - H, stage, mid, stage);
  float m[kFP];
#pragma unroll
  for (int p = 0; p < kFP; ++p) {
    int li, lj;
    float w1[4], w2[4];
    box_stencil<W>(H + cx + kFS * p, H + r, x1[p], x2[p], false, li, lj, w1, w2);
    m[p] = apply_box<D::PB>(stage, li, lj, w1, w2);
    m[p] -= 0.5f * ht * (w1v[p] * G1[p] + w2v[p] * G2[p] + u1[p] * g1[p] + u2[p] * g2[p]);
  }
  if (!b) {
    stf(out + idx, m);
    return;
  }
  float gn1[kFP], gn2[kFP], lam[kFP], b1[kFP], b2[kFP];
  ldf(gm_nt + idx, gn1);
  ldf(gm_nt + N + idx, gn2);
  const float hh = 0.5f * ht;
#pragma unroll
  for (int p = 0; p < kFP; ++p) {
    lam[p] = -m[p];
    b1[p] = hh * lam[p] * gn1[p];
    b2[p] = hh * lam[p] * gn2[p];
  }
  stf(out + idx, lam);
  stf(b + idx, b1);
  stf(b + N + idx, b2);
}

template <bool P2, int W>
__global__ void __launch_bounds__(kFT, 2)
k_incstate_fused(int n1, int n2, int log1, float ht, const float* __restrict__ m_prev,
                 const float* __restrict__ dX, const float* __restrict__ vt,
                 const float* __restrict__ vtD, const float* __restrict__ G,
                 const float* __restrict__ gm, float* __restrict__ out,
                 const float* __restrict__ gm_nt, float* __restrict__ b) {
  pdl_enter();
  extern __shared__ float sm[];
  incstate_fused_body<P2, W>(n1, n2, log1, blockIdx.x * 32, blockIdx.y * 32, sm, ht, m_prev, dX,
                             vt, vtD, G, gm, out, gm_nt, b);
}

// v~ at the departure points and the first incremental state step in one
// kernel: both components of v~ are prefiltered on the tile's box, gathered
// at X_D (written to vtD, needed by every later step) and
// m~_1 = -h_t/2 (v~(X_D) . grad m_0(X_D) + v~ . grad m_1) (m~_0 = 0).
template <bool P2, int W>
__device__ __forceinline__ void incstate_first_fused_body(
    int n1, int n2, int log1, int x0, int y0, float* sm, float ht, const float* __restrict__ vt,
    const float* __restrict__ dX, const float* __restrict__ G1p, const float* __restrict__ gm1,
    float* __restrict__ vtD, float* __restrict__ out) {
  using D = BoxDims<W>;
  constexpr int H = (W - 32) / 2;
  constexpr int kBox = W * D::PB;
  float* stage = sm;
  float* mid = sm + D::kStage;
  float* box1 = mid + D::kMid;
  const long long N = (long long)n1 * n2;
  constexpr int TPR = 32 / kFP;
  const int t = threadIdx.x, r = t / TPR, cx = t % TPR;
  const long long idx = row_offset<P2>(y0 + r, n1, log1) + x0 + cx;
  // (the streamed operands are loaded after the two prefilters: loading
  // them first took more registers than two blocks per SM allow)
  prefilter_box<W, P2, kFT>(vt, n1, n2, log1, x0 - H, y0 - H, stage, mid, box1);
  prefilter_box<W, P2, kFT>(vt + N, n1, n2, log1, x0 - H, y0 - H, stage, mid, stage);
  (void)kBox;
  float x1[kFP], x2[kFP], Ga[kFP], Gb[kFP], u1[kFP], u2[kFP], g1[kFP], g2[kFP];
  ldf(dX + idx, x1);
  ldf(dX + N + idx, x2);
  ldf(G1p + idx, Ga);
  ldf(G1p + N + idx, Gb);
  ldf(vt + idx, u1);
  ldf(vt + N + idx, u2);
  ldf(gm1 + idx, g1);
  ldf(gm1 + N + idx, g2);
  float wd1[kFP], wd2[kFP], m[kFP];
#pragma unroll
  for (int p = 0; p < kFP; ++p) {
    int li, lj;
    float w1[4], w2[4];
    box_stencil<W>(H + cx + kFS * p, H + r, x1[p], x2[p], false, li, lj, w1, w2);
    wd1[p] = apply_box<D::PB>(box1, li, lj, w1, w2);
    wd2[p] = apply_box<D::PB>(stage, li, lj, w1, w2);
    m[p] = 0.f;
    m[p] -= 0.5f * ht * (wd1[p] * Ga[p] + wd2[p] * Gb[p] + u1[p] * g1[p] + u2[p] * g2[p]);
  }
  stf(vtD + idx, wd1);
  stf(vtD + N + idx, wd2);
  stf(out + idx, m);
}

template <bool P2, int W>
__global__ void __launch_bounds__(kFT, 2)
k_incstate_first_fused(int n1, int n2, int log1, float ht, const float* __restrict__ vt,
                       const float* __restrict__ dX, const float* __restrict__ G1p,
                       const float* __restrict__ gm1, float* __restrict__ vtD,
                       float* __restrict__ out) {
  pdl_enter();
  extern __shared__ float sm[];
  incstate_first_fused_body<P2, W>(n1, n2, log1, blockIdx.x * 32, blockIdx.y * 32, sm, ht, vt, dX,
                                   G1p, gm1, vtD, out);
}

// Prefilter + gather of F = 1 or 2 fields (fstride apart) at the departure
// points disp, on the tile's box: the state step m_j = m_{j-1}(X_D) and the
// history G_j = grad m_{j-1}(X_D) without a coefficient field in memory.
template <bool P2, int W, int F>
__device__ __forceinline__ void gather_fused_body(int n1, int n2, int log1, int x0, int y0,
                                                  float* sm, const float* __restrict__ u,
                                                  long long fstride,
                                                  const float* __restrict__ disp,
                                                  float* __restrict__ out) {
  using D = BoxDims<W>;
  constexpr int H = (W - 32) / 2;
  float* stage = sm;
  float* mid = sm + D::kStage;
  float* box1 = mid + D::kMid;     // first field's box when F = 2
  const long long N = (long long)n1 * n2;
  constexpr int TPR = 32 / kFP;
  const int t = threadIdx.x, r = t / TPR, cx = t % TPR;
  const long long idx = row_offset<P2>(y0 + r, n1, log1) + x0 + cx;
  float d1[kFP], d2[kFP];
  ldf(disp + idx, d1);
  ldf(disp + N + idx, d2);
  if (F == 2)
    prefilter_box<W, P2, kFT>(u, n1, n2, log1, x0 - H, y0 - H, stage, mid, box1);
  prefilter_box<W, P2, kFT>(u + (F - 1) * fstride, n1, n2, log1, x0 - H, y0 - H, stage, mid, stage);
  float o1[kFP], o2[kFP];
#pragma unroll
  for (int p = 0; p < kFP; ++p) {
    int li, lj;
    float w1[4], w2[4];
    box_stencil<W>(H + cx + kFS * p, H + r, d1[p], d2[p], false, li, lj, w1, w2);
    if (F == 2) o1[p] = apply_box<D::PB>(box1, li, lj, w1, w2);
    o2[p] = apply_box<D::PB>(stage, li, lj, w1, w2);
  }
  if (F == 2) {
    stf(out + idx, o1);
    stf(out + fstride + idx, o2);
  } else {
    stf(out + idx, o2);
  }
}

template <bool P2, int W, int F>
__global__ void __launch_bounds__(kFT, 2)
k_gather_fused(int n1, int n2, int log1, const float* __restrict__ u, long long fstride,
               const float* __restrict__ disp, float* __restrict__ out) {
  pdl_enter();
  extern __shared__ float sm[];
  gather_fused_body<P2, W, F>(n1, n2, log1, blockIdx.x * 32, blockIdx.y * 32, sm, u, fstride,
                              disp, out);
}

// box widths with a fused kernel: halo H = 8 and H = 16
constexpr int kFuseW[2] = {48, 64};

int fused_box_width(double max_disp_cells) {
  for (int W : kFuseW)
    if (max_disp_cells <= (double)((W - 32) / 2 - 2)) return W;
  return 0;
}

template <typename K>
static void allow_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int W>
constexpr size_t first_smem() {
  return BoxDims<W>::kSmemBytes + sizeof(float) * W * BoxDims<W>::PB;
}

void fused_init() {
  allow_smem(k_gather_fused<true, 48, 1>, BoxDims<48>::kSmemBytes);
  allow_smem(k_gather_fused<false, 48, 1>, BoxDims<48>::kSmemBytes);
  allow_smem(k_gather_fused<true, 64, 1>, BoxDims<64>::kSmemBytes);
  allow_smem(k_gather_fused<false, 64, 1>, BoxDims<64>::kSmemBytes);
  allow_smem(k_gather_fused<true, 48, 2>, first_smem<48>());
  allow_smem(k_gather_fused<false, 48, 2>, first_smem<48>());
  allow_smem(k_gather_fused<true, 64, 2>, first_smem<64>());
  allow_smem(k_gather_fused<false, 64, 2>, first_smem<64>());
  allow_smem(k_incstate_first_fused<true, 48>, first_smem<48>());
  allow_smem(k_incstate_first_fused<false, 48>, first_smem<48>());
  allow_smem(k_incstate_first_fused<true, 64>, first_smem<64>());
  allow_smem(k_incstate_first_fused<false, 64>, first_smem<64>());
  allow_smem(k_adjoint_fused<true, 48>, BoxDims<48>::kSmemBytes);
  allow_smem(k_adjoint_fused<false, 48>, BoxDims<48>::kSmemBytes);
  allow_smem(k_adjoint_fused<true, 64>, BoxDims<64>::kSmemBytes);
  allow_smem(k_adjoint_fused<false, 64>, BoxDims<64>::kSmemBytes);
  allow_smem(k_incstate_fused<true, 48>, BoxDims<48>::kSmemBytes);
  allow_smem(k_incstate_fused<false, 48>, BoxDims<48>::kSmemBytes);
  allow_smem(k_incstate_fused<true, 64>, BoxDims<64>::kSmemBytes);
  allow_smem(k_incstate_fused<false, 64>, BoxDims<64>::kSmemBytes);
}

void launch_adjoint_fused(int W, int n1, int n2, float ht, float wb, const float* lam_next,
                          const float* dY, const float* delta, const float* delta_bar,
                          const float* gm, float* lam_out, float* b, cudaStream_t st) {
  const dim3 grid(n1 / 32, n2 / 32);
  const bool p2 = pow2_grid(n1, n2);
  if (W == 48)
    launch_k(p2 ? k_adjoint_fused<true, 48> : k_adjoint_fused<false, 48>, grid, dim3(kFT),
             BoxDims<48>::kSmemBytes, st, n1, n2, ilog2i(n1), ht, wb, lam_next, dY, delta, delta_bar,
             gm, lam_out, b);
  else
    launch_k(p2 ? k_adjoint_fused<true, 64> : k_adjoint_fused<false, 64>, grid, dim3(kFT),
             BoxDims<64>::kSmemBytes, st, n1, n2, ilog2i(n1), ht, wb, lam_next, dY, delta, delta_bar,
             gm, lam_out, b);
}

void launch_incstate_fused(int W, int n1, int n2, float ht, const float* m_prev, const float* dX,
                           const float* vt, const float* vtD, const float* G, const float* gm,
                           float* out, const float* gm_nt, float* b, cudaStream_t st) {
  const dim3 grid(n1 / 32, n2 / 32);
  const bool p2 = pow2_grid(n1, n2);
  if (W == 48)
    launch_k(p2 ? k_incstate_fused<true, 48> : k_incstate_fused<false, 48>, grid, dim3(kFT),
             BoxDims<48>::kSmemBytes, st, n1, n2, ilog2i(n1), ht, m_prev, dX, vt, vtD, G, gm, out,
             gm_nt, b);
  else
    launch_k(p2 ? k_incstate_fused<true, 64> : k_incstate_fused<false, 64>, grid, dim3(kFT),
             BoxDims<64>::kSmemBytes, st, n1, n2, ilog2i(n1), ht, m_prev, dX, vt, vtD, G, gm, out,
             gm_nt, b);
}

void launch_incstate_first_fused(int W, int n1, int n2, float ht, const float* vt, const float* dX,
                                 const float* G1, const float* gm1, float* vtD, float* out,
                                 cudaStream_t st) {
  const dim3 grid(n1 / 32, n2 / 32);
  const bool p2 = pow2_grid(n1, n2);
  if (W == 48)
    launch_k(p2 ? k_incstate_first_fused<true, 48> : k_incstate_first_fused<false, 48>, grid,
             dim3(kFT), first_smem<48>(), st, n1, n2, ilog2i(n1), ht, vt, dX, G1, gm1, vtD, out);
  else
    launch_k(p2 ? k_incstate_first_fused<true, 64> : k_incstate_first_fused<false, 64>, grid,
             dim3(kFT), first_smem<64>(), st, n1, n2, ilog2i(n1), ht, vt, dX, G1, gm1, vtD, out);
}

void launch_gather_fused(int W, int n1, int n2, const float* u, long long fstride, int F,
                         const float* disp, float* out, cudaStream_t st) {
  const dim3 grid(n1 / 32, n2 / 32);
  const bool p2 = pow2_grid(n1, n2);
  const int lg = ilog2i(n1);
#define REGNK_GF(WW, FF, SM)                                                                    \
  launch_k(p2 ? k_gather_fused<true, WW, FF> : k_gather_fused<false, WW, FF>, grid, dim3(kFT), \
           SM, st, n1, n2, lg, u, fstride, disp, out)
  if (W == 48 && F == 1) REGNK_GF(48, 1, BoxDims<48>::kSmemBytes);
  else if (W == 48) REGNK_GF(48, 2, first_smem<48>());
  else if (F == 1) REGNK_GF(64, 1, BoxDims<64>::kSmemBytes);
  else REGNK_GF(64, 2, first_smem<64>());
#undef REGNK_GF
}

// ---------------------------------------------------------------------------
// Batched kernels: the same per-tile and per-point bodies over the tiles of
// every problem of a batch in one launch (see BatchView). A tile block reads
// its problem and tile from the table, skips problems outside the mask and
// problems whose displacements exceed the fused kernels' halo (w = 0), and
// runs the body for the problem's index arithmetic (power-of-two grid or
// not) and box width, so each problem's results are bitwise those of the
// one-problem kernels.

__device__ __forceinline__ float* bref(const BRef& r, const BDesc& D) {
  return r.base ? r.base + (long long)r.F * D.off + (long long)r.k * D.n1 * D.n2 : nullptr;
}

template <bool V>
using BoolC = std::integral_constant<bool, V>;
template <int V>
using IntC = std::integral_constant<int, V>;

// fn(P2, W) with both as compile-time constants
template <typename Fn>
__device__ __forceinline__ void by_shape(const BDesc& D, int W, Fn fn) {
  if (D.p2) {
    if (W == 48) fn(BoolC<true>{}, IntC<48>{});
    else fn(BoolC<true>{}, IntC<64>{});
  } else {
    if (W == 48) fn(BoolC<false>{}, IntC<48>{});
    else fn(BoolC<false>{}, IntC<64>{});
  }
}

// The block's problem and tile origin; false if the block has nothing to do.
__device__ __forceinline__ bool batch_tile(const BatchView& B, bool need_w, BDesc& D, int& W,
                                           int& x0, int& y0) {
  const int4 tj = B.tiles[blockIdx.x];
  if (!B.mask[tj.x]) return false;
  D = B.desc[tj.x];
  W = need_w ? B.w[tj.x] : 48;
  x0 = tj.y * 32;
  y0 = tj.z * 32;
  return W != 0;
}

// one block per tile and field (blockIdx.y)
__global__ void __launch_bounds__(kPThreads)
k_prefilter_b(BatchView B, BRef in, BRef out) {
  pdl_enter();
  __shared__ float sin_[kPH * kPIn];
  __shared__ float smid[kPH * kPMid];
  BDesc D;
  int W, x0, y0;
  if (!batch_tile(B, false, D, W, x0, y0)) return;
  in.k += blockIdx.y;
  out.k += blockIdx.y;
  const float* src = bref(in, D);
  float* dst = bref(out, D);
  if (D.p2) prefilter_tile<true>(src, dst, D.n1, D.n2, D.log1, x0, y0, sin_, smid);
  else prefilter_tile<false>(src, dst, D.n1, D.n2, D.log1, x0, y0, sin_, smid);
}

void launch_prefilter_b(const BatchView& B, BRef in, BRef out, int F, cudaStream_t st) {
  launch_k(k_prefilter_b, dim3(B.ntiles, F), dim3(kPThreads), 0, st, B, in, out);
}

// one thread per point of the batch
__global__ void __launch_bounds__(kPT)
k_departure_b(BatchView B, long long npts, BRef v, BRef cv, BRef dX, BRef dY) {
  pdl_enter();
  const long long g = (long long)blockIdx.x * kPT + threadIdx.x;
  if (g >= npts) return;
  const int p = B.pmap[g >> 10];
  if (!B.mask[p]) return;
  const BDesc D = B.desc[p];
  const long long idx = g - D.off;
  if (D.p2)
    departure_point<true>(idx, D.n1, D.n2, D.log1, D.s1, D.s2, bref(v, D), bref(cv, D),
                          bref(dX, D), bref(dY, D), 0);
  else
    departure_point<false>(idx, D.n1, D.n2, D.log1, D.s1, D.s2, bref(v, D), bref(cv, D),
                           bref(dX, D), bref(dY, D), 0);
}

void launch_departure_b(const BatchView& B, long long npts, BRef v, BRef cv, BRef dX, BRef dY,
                        cudaStream_t st) {
  launch_k(k_departure_b, dim3((unsigned)((npts + kPT - 1) / kPT)), dim3(kPT), 0, st, B, npts, v,
           cv, dX, dY);
}

// w_p from the largest displacements of X_D and Y_D, the rule of
// fused_box_width
__global__ void k_set_w_b(int nprob, const double* __restrict__ dmax_x,
                          const double* __restrict__ dmax_y, int* __restrict__ w) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  const double d = fmax(dmax_x[p], dmax_y[p]);
  int W = 0;
  if (d <= (double)((48 - 32) / 2 - 2)) W = 48;
  else if (d <= (double)((64 - 32) / 2 - 2)) W = 64;
  w[p] = W;
}

void launch_set_w_b(int nprob, const double* dmax_x, const double* dmax_y, int* w,
                    cudaStream_t st) {
  launch_k(k_set_w_b, dim3((nprob + 127) / 128), dim3(128), 0, st, nprob, dmax_x, dmax_y, w);
}

__global__ void __launch_bounds__(kPT)
k_adjoint_init_b(BatchView B, long long npts, float coef_b, BRef mR, BRef m1, BRef gm, BRef lam,
                 BRef b, float sign) {
  pdl_enter();
  const long long g = (long long)blockIdx.x * kPT + threadIdx.x;
  if (g >= npts) return;
  const int p = B.pmap[g >> 10];
  if (!B.mask[p]) return;
  const BDesc D = B.desc[p];
  adjoint_init_point(g - D.off, (long long)D.n1 * D.n2, coef_b, bref(mR, D), bref(m1, D),
                     bref(gm, D), bref(lam, D), bref(b, D), sign);
}

void launch_adjoint_init_b(const BatchView& B, long long npts, float coef_b, BRef mR, BRef m1,
                           BRef gm, BRef lam, BRef b, float sign, cudaStream_t st) {
  launch_k(k_adjoint_init_b, dim3((unsigned)((npts + kPT - 1) / kPT)), dim3(kPT), 0, st, B, npts,
           coef_b, mR, m1, gm, lam, b, sign);
}

// dst = src, one scalar field per problem (e.g. m_0 = m_T into the history)
__global__ void __launch_bounds__(kPT)
k_copy_field_b(BatchView B, long long npts, BRef src, BRef dst) {
  pdl_enter();
  const long long g = (long long)blockIdx.x * kPT + threadIdx.x;
  if (g >= npts) return;
  const int p = B.pmap[g >> 10];
  if (!B.mask[p]) return;
  const BDesc D = B.desc[p];
  bref(dst, D)[g - D.off] = __ldg(bref(src, D) + (g - D.off));
}

void launch_copy_field_b(const BatchView& B, long long npts, BRef src, BRef dst, cudaStream_t st) {
  launch_k(k_copy_field_b, dim3((unsigned)((npts + kPT - 1) / kPT)), dim3(kPT), 0, st, B, npts, src,
           dst);
}

template <int F>
__global__ void __launch_bounds__(kFT, 2)
k_gather_fused_b(BatchView B, BRef u, BRef disp, BRef out) {
  pdl_enter();
  extern __shared__ float sm[];
  BDesc D;
  int W, x0, y0;
  if (!batch_tile(B, true, D, W, x0, y0)) return;
  const long long N = (long long)D.n1 * D.n2;
  by_shape(D, W, [&](auto P2, auto WC) {
    gather_fused_body<decltype(P2)::value, decltype(WC)::value, F>(
        D.n1, D.n2, D.log1, x0, y0, sm, bref(u, D), N, bref(disp, D), bref(out, D));
  });
}

__global__ void __launch_bounds__(kFT, 2)
k_adjoint_fused_b(BatchView B, float ht, float wb, BRef lam_next, BRef dY, BRef delta,
                  BRef delta_bar, BRef gm, BRef lam_out, BRef b) {
  pdl_enter();
  extern __shared__ float sm[];
  BDesc D;
  int W, x0, y0;
  if (!batch_tile(B, true, D, W, x0, y0)) return;
  by_shape(D, W, [&](auto P2, auto WC) {
    adjoint_fused_body<decltype(P2)::value, decltype(WC)::value>(
        D.n1, D.n2, D.log1, x0, y0, sm, ht, wb, bref(lam_next, D), bref(dY, D), bref(delta, D),
        bref(delta_bar, D), bref(gm, D), bref(lam_out, D), bref(b, D));
  });
}

__global__ void __launch_bounds__(kFT, 2)
k_incstate_first_fused_b(BatchView B, float ht, BRef vt, BRef dX, BRef G1, BRef gm1, BRef vtD,
                         BRef out) {
  pdl_enter();
  extern __shared__ float sm[];
  BDesc D;
  int W, x0, y0;
  if (!batch_tile(B, true, D, W, x0, y0)) return;
  by_shape(D, W, [&](auto P2, auto WC) {
    incstate_first_fused_body<decltype(P2)::value, decltype(WC)::value>(
        D.n1, D.n2, D.log1, x0, y0, sm, ht, bref(vt, D), bref(dX, D), bref(G1, D), bref(gm1, D),
        bref(vtD, D), bref(out, D));
  });
}

__global__ void __launch_bounds__(kFT, 2)
k_incstate_fused_b(BatchView B, float ht, BRef m_prev, BRef dX, BRef vt, BRef vtD, BRef G,
                   BRef gm, BRef out, BRef gm_nt, BRef b) {
  pdl_enter();
  extern __shared__ float sm[];
  BDesc D;
  int W, x0, y0;
  if (!batch_tile(B, true, D, W, x0, y0)) return;
  by_shape(D, W, [&](auto P2, auto WC) {
    incstate_fused_body<decltype(P2)::value, decltype(WC)::value>(
        D.n1, D.n2, D.log1, x0, y0, sm, ht, bref(m_prev, D), bref(dX, D), bref(vt, D),
        bref(vtD, D), bref(G, D), bref(gm, D), bref(out, D), bref(gm_nt, D), bref(b, D));
  });
}

// shared memory of the batched fused kernels: the 64^2 box (any problem may need it)
void batch_fused_init() {
  allow_smem(k_gather_fused_b<1>, BoxDims<64>::kSmemBytes);
  allow_smem(k_gather_fused_b<2>, first_smem<64>());
  allow_smem(k_incstate_first_fused_b, first_smem<64>());
  allow_smem(k_adjoint_fused_b, BoxDims<64>::kSmemBytes);
  allow_smem(k_incstate_fused_b, BoxDims<64>::kSmemBytes);
}

void launch_gather_fused_b(const BatchView& B, BRef u, int F, BRef disp, BRef out,
                           cudaStream_t st) {
  if (F == 2)
    launch_k(k_gather_fused_b<2>, dim3(B.ntiles), dim3(kFT), first_smem<64>(), st, B, u, disp, out);
  else
    launch_k(k_gather_fused_b<1>, dim3(B.ntiles), dim3(kFT), BoxDims<64>::kSmemBytes, st, B, u,
             disp, out);
}

void launch_adjoint_fused_b(const BatchView& B, float ht, float wb, BRef lam_next, BRef dY,
                            BRef delta, BRef delta_bar, BRef gm, BRef lam_out, BRef b,
                            cudaStream_t st) {
  launch_k(k_adjoint_fused_b, dim3(B.ntiles), dim3(kFT), BoxDims<64>::kSmemBytes, st, B, ht, wb,
           lam_next, dY, delta, delta_bar, gm, lam_out, b);
}

void launch_incstate_first_fused_b(const BatchView& B, float ht, BRef vt, BRef dX, BRef G1,
                                   BRef gm1, BRef vtD, BRef out, cudaStream_t st) {
  launch_k(k_incstate_first_fused_b, dim3(B.ntiles), dim3(kFT), first_smem<64>(), st, B, ht, vt,
           dX, G1, gm1, vtD, out);
}

void launch_incstate_fused_b(const BatchView& B, float ht, BRef m_prev, BRef dX, BRef vt,
                             BRef vtD, BRef G, BRef gm, BRef out, BRef gm_nt, BRef b,
                             cudaStream_t st) {
  launch_k(k_incstate_fused_b, dim3(B.ntiles), dim3(kFT), BoxDims<64>::kSmemBytes, st, B, ht,
           m_prev, dX, vt, vtD, G, gm, out, gm_nt, b);
}

}  // namespace regnk
