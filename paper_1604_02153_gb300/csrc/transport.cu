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

#include "common.cuh"
#include "interp.cuh"
#include "kernels.h"

namespace regnk {

// One block per 32x32 output tile and field.
__global__ void __launch_bounds__(kPThreads)
k_prefilter(const float* __restrict__ in, float* __restrict__ out, int n1, int n2, int log1,
            long long fstride) {
  __shared__ float sin_[kPH * kPIn];
  __shared__ float smid[kPH * kPMid];
  const long long fo = (long long)blockIdx.z * fstride;
  prefilter_tile(in + fo, out + fo, n1, n2, log1, blockIdx.x * kPX, blockIdx.y * kPY, sin_,
                 smid);
}

static int ilog2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

void launch_prefilter(int n1, int n2, const float* in, float* tmp, float* out, int F,
                      cudaStream_t st) {
  (void)tmp;
  k_prefilter<<<dim3(n1 / kPX, n2 / kPY, F), kPThreads, 0, st>>>(in, out, n1, n2, ilog2i(n1),
                                                                  (long long)n1 * n2);
  ++g_launch_count;
}

constexpr int kPT = 256;  // threads per block of the pointwise kernels

// Departure points of both characteristics (Heun, §3.3.2):
//   X* = x - h_t v(x),  X_D = x - h_t/2 (v(x) + v(X*))
//   Y* = x + h_t v(x),  Y_D = x + h_t/2 (v(x) + v(Y*))
// cv holds the interpolation coefficients of v (spline) or v itself.
__global__ void __launch_bounds__(kPT)
k_departure(int n1, int n2, int log1, float s1, float s2, const float* __restrict__ v,
            const float* __restrict__ cv, float* __restrict__ dX, float* __restrict__ dY,
            int lagrange) {
  const long long N = (long long)n1 * n2;
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  const int i = (int)(idx & (n1 - 1)), j = (int)(idx >> log1);
  const float v1 = __ldg(v + idx), v2 = __ldg(v + N + idx);
  const float a1 = s1 * v1, a2 = s2 * v2;   // h_t v / h in cells
  if (dX) {
    const Stencil S = make_stencil(i, j, -a1, -a2, n1, n2, log1, lagrange);
    const float w1 = apply_stencil(S, cv), w2 = apply_stencil(S, cv + N);
    dX[idx] = -0.5f * (a1 + s1 * w1);
    dX[N + idx] = -0.5f * (a2 + s2 * w2);
  }
  if (dY) {
    const Stencil S = make_stencil(i, j, a1, a2, n1, n2, log1, lagrange);
    const float w1 = apply_stencil(S, cv), w2 = apply_stencil(S, cv + N);
    dY[idx] = 0.5f * (a1 + s1 * w1);
    dY[N + idx] = 0.5f * (a2 + s2 * w2);
  }
}

void launch_departure(int n1, int n2, float ht, const float* v, const float* cv, float* dX,
                      float* dY, int lagrange, cudaStream_t st) {
  const long long N = (long long)n1 * n2;
  const float s1 = ht * n1 / (2.0f * 3.14159265358979323846f);
  const float s2 = ht * n2 / (2.0f * 3.14159265358979323846f);
  k_departure<<<(unsigned)((N + kPT - 1) / kPT), kPT, 0, st>>>(n1, n2, ilog2i(n1), s1, s2, v,
                                                                cv, dX, dY, lagrange); ++g_launch_count;
}

// out_f = I[coef_f](x + disp), f = 0..F-1 (fields fstride apart), one stencil.
__global__ void __launch_bounds__(kPT)
k_gather(int n1, int n2, int log1, const float* __restrict__ coef,
         const float* __restrict__ disp, float* __restrict__ out, int F, long long fstride,
         int lagrange) {
  const long long N = (long long)n1 * n2;
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  const int i = (int)(idx & (n1 - 1)), j = (int)(idx >> log1);
  const Stencil S = make_stencil(i, j, __ldg(disp + idx), __ldg(disp + N + idx), n1, n2, log1,
                                 lagrange);
  for (int f = 0; f < F; ++f) out[f * fstride + idx] = apply_stencil(S, coef + f * fstride);
}

void launch_gather(int n1, int n2, const float* coef, const float* disp, float* out, int F,
                   long long fstride, int lagrange, cudaStream_t st) {
  const long long N = (long long)n1 * n2;
  k_gather<<<(unsigned)((N + kPT - 1) / kPT), kPT, 0, st>>>(n1, n2, ilog2i(n1), coef, disp,
                                                             out, F, fstride, lagrange); ++g_launch_count;
}

void launch_state_step(int n1, int n2, const float* coef, const float* dX, float* out,
                       int lagrange, cudaStream_t st) {
  launch_gather(n1, n2, coef, dX, out, 1, 0, lagrange, st);
}

// Final condition of an adjoint solve and the first term of its time
// integral: lam = sign * (mR - m1) (mR may be NULL: lam = -sign * m1),
// b = coef_b * lam * grad m.
__global__ void __launch_bounds__(kPT)
k_adjoint_init(long long N, float coef_b, const float* __restrict__ mR,
               const float* __restrict__ m1, const float* __restrict__ gm,
               float* __restrict__ lam, float* __restrict__ b, float sign) {
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  const float r = (mR ? __ldg(mR + idx) : 0.f) - __ldg(m1 + idx);
  const float l = sign * r;
  lam[idx] = l;
  b[idx] = coef_b * l * __ldg(gm + idx);
  b[N + idx] = coef_b * l * __ldg(gm + N + idx);
}

void launch_adjoint_init(int n1, int n2, float coef_b, const float* mR, const float* m1,
                         const float* gm, float* lam, float* b, float sign, cudaStream_t st) {
  const long long N = (long long)n1 * n2;
  k_adjoint_init<<<(unsigned)((N + kPT - 1) / kPT), kPT, 0, st>>>(N, coef_b, mR, m1, gm, lam,
                                                                  b, sign); ++g_launch_count;
}

// One backward step of the (incremental) adjoint along Y_D (§3.3.2, Heun):
//   lb = lam_{j+1}(Y_D), lam* = lb + h_t lb div v(Y_D),
//   lam_j = lb + h_t/2 (lb div v(Y_D) + lam* div v(x)),
// fused with the time integral b += wb * lam_j * grad m_j.
__global__ void __launch_bounds__(kPT)
k_adjoint_step(int n1, int n2, int log1, float ht, float wb, const float* __restrict__ coef,
               const float* __restrict__ dY, const float* __restrict__ delta,
               const float* __restrict__ delta_bar, const float* __restrict__ gm,
               float* __restrict__ lam_out, float* __restrict__ b, int lagrange) {
  const long long N = (long long)n1 * n2;
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  const int i = (int)(idx & (n1 - 1)), j = (int)(idx >> log1);
  const Stencil S = make_stencil(i, j, __ldg(dY + idx), __ldg(dY + N + idx), n1, n2, log1,
                                 lagrange);
  const float lb = apply_stencil(S, coef);
  const float db = __ldg(delta_bar + idx), d = __ldg(delta + idx);
  const float lstar = fmaf(ht * lb, db, lb);
  const float l = lb + 0.5f * ht * (lb * db + lstar * d);
  lam_out[idx] = l;
  b[idx] = fmaf(wb * l, __ldg(gm + idx), b[idx]);
  b[N + idx] = fmaf(wb * l, __ldg(gm + N + idx), b[N + idx]);
}

void launch_adjoint_step(int n1, int n2, float ht, float wb, const float* coef,
                         const float* dY, const float* delta, const float* delta_bar,
                         const float* gm, float* lam_out, float* b, int lagrange,
                         cudaStream_t st) {
  const long long N = (long long)n1 * n2;
  k_adjoint_step<<<(unsigned)((N + kPT - 1) / kPT), kPT, 0, st>>>(
      n1, n2, ilog2i(n1), ht, wb, coef, dY, delta, delta_bar, gm, lam_out, b, lagrange); ++g_launch_count;
}

// One forward step of the incremental state (Gauss-Newton, §3.3.2):
//   m~_j = m~_{j-1}(X_D) - h_t/2 (v~(X_D) . grad m_{j-1}(X_D) + v~ . grad m_j)
// G = grad m_{j-1}(X_D) (2 fields), vtD = v~(X_D) (2 fields), gm = grad m_j.
// first = 1 for j = 1 where m~_0 = 0.
__global__ void __launch_bounds__(kPT)
k_incstate_step(int n1, int n2, int log1, float ht, const float* __restrict__ coef,
                const float* __restrict__ dX, const float* __restrict__ vt,
                const float* __restrict__ vtD, const float* __restrict__ G,
                const float* __restrict__ gm, float* __restrict__ out, int first,
                int lagrange) {
  const long long N = (long long)n1 * n2;
  const long long idx = (long long)blockIdx.x * kPT + threadIdx.x;
  if (idx >= N) return;
  float base = 0.f;
  if (!first) {
    const int i = (int)(idx & (n1 - 1)), j = (int)(idx >> log1);
    const Stencil S = make_stencil(i, j, __ldg(dX + idx), __ldg(dX + N + idx), n1, n2, log1,
                                   lagrange);
    base = apply_stencil(S, coef);
  }
  const float src_dep = __ldg(vtD + idx) * __ldg(G + idx) + __ldg(vtD + N + idx) * __ldg(G + N + idx);
  const float src_arr = __ldg(vt + idx) * __ldg(gm + idx) + __ldg(vt + N + idx) * __ldg(gm + N + idx);
  out[idx] = base - 0.5f * ht * (src_dep + src_arr);
}

void launch_incstate_step(int n1, int n2, float ht, const float* coef, const float* dX,
                          const float* vt, const float* vtD, const float* G, const float* gm,
                          float* out, int first, int lagrange, cudaStream_t st) {
  const long long N = (long long)n1 * n2;
  k_incstate_step<<<(unsigned)((N + kPT - 1) / kPT), kPT, 0, st>>>(
      n1, n2, ilog2i(n1), ht, coef, dX, vt, vtD, G, gm, out, first, lagrange); ++g_launch_count;
}

}  // namespace regnk
