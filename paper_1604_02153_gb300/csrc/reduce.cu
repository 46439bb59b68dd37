// Reductions and Krylov vector updates. Inner products and norms take FP32
// fields and are accumulated to FP64 accuracy (the Krylov inner products, the
// Armijo objective comparison and the gradient-norm test of §3.4.1 are
// decided in FP64). Each thread carries its partial sum as an unevaluated
// pair of FP32 numbers built with error-free transformations (FMA-based
// TwoProduct for a*b, TwoSum for each addition, TwoDiff for a-b), so every
// product and difference enters exactly and only second-order rounding is
// lost; the pair is converted to FP64 once per thread and the block and
// final sums are FP64. This keeps the FP64 pipe (a small fraction of the
// FP32 rate on this GPU) off the per-element path. Reductions are two-stage
// with a fixed block count and a fixed summation order, so repeated calls on
// the same data give identical bits.
#include "common.cuh"
#include "kernels.h"

namespace regnk {

constexpr int kRT = 256;       // threads per reduction block
constexpr int kRB = 1216;      // maximum partial sums (8 per SM on 152 SMs)

int reduce_partials() { return kRB; }
static_assert(kRT == 256 && kRB == 1216, "reduce_blocks (kernels.h) assumes these");

static int nblocks(long long n) {
  long long b = (n + 4LL * kRT - 1) / (4LL * kRT);
  return (int)(b < 1 ? 1 : (b > kRB ? kRB : b));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v) {
  __shared__ T ws[kRT / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  T r = 0;
  if (w == 0) {
    r = lane < kRT / 32 ? ws[lane] : T(0);
    r = warp_sum(r);
  }
  return r;
}

// FP32 pair (s, c) accumulating a sum with Knuth's TwoSum: s + c carries the
// exact sum up to second-order rounding terms.
struct Pair {
  float s = 0.f, c = 0.f;
};
__device__ __forceinline__ void pair_add(Pair& a, float p) {
  const float t = a.s + p;
  const float z = t - a.s;
  a.c += (a.s - (t - z)) + (p - z);
  a.s = t;
}
// adds x*y (MODE 0) or (x-y)^2 (MODE 1) exactly up to second-order terms
template <int MODE>
__device__ __forceinline__ void pair_term(Pair& a, float x, float y) {
  if (MODE == 0) {
    const float p = x * y;
    pair_add(a, p);
    a.c += fmaf(x, y, -p);                  // exact rounding error of x*y
  } else {
    const float d = x - y;
    const float z = d - x;
    const float dd = (x - (d - z)) + (-y - z);   // exact rounding error of x-y
    const float p = d * d;
    pair_add(a, p);
    a.c += fmaf(d, d, -p) + 2.f * d * dd;   // (d+dd)^2 = d^2 + 2 d dd + dd^2
  }
}

// Block `bi` of `nblk` of the two-stage sum over n values: mode 0: sum
// a*b; mode 1: sum (a-b)^2. The result is valid in thread 0.
template <int MODE>
__device__ __forceinline__ double partial_sum(const float* __restrict__ a,
                                              const float* __restrict__ b, long long n, int nblk,
                                              int bi, int vec4) {
  Pair acc;
  const long long stride = (long long)nblk * kRT;
  const long long n4 = vec4 ? (n >> 2) : 0;   // float4 path only for 16-byte aligned inputs
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
#pragma unroll 4
  for (long long i = (long long)bi * kRT + threadIdx.x; i < n4; i += stride) {
    const float4 x = __ldg(a4 + i), y = __ldg(b4 + i);
    pair_term<MODE>(acc, x.x, y.x);
    pair_term<MODE>(acc, x.y, y.y);
    pair_term<MODE>(acc, x.z, y.z);
    pair_term<MODE>(acc, x.w, y.w);
  }
  for (long long i = (n4 << 2) + (long long)bi * kRT + threadIdx.x; i < n; i += stride)
    pair_term<MODE>(acc, __ldg(a + i), __ldg(b + i));
  return block_sum((double)acc.s + (double)acc.c);
}

template <int MODE>
__global__ void __launch_bounds__(kRT)
k_partial(const float* __restrict__ a, const float* __restrict__ b, long long n,
          double* __restrict__ partial, int vec4) {
  pdl_enter();
  const double s = partial_sum<MODE>(a, b, n, gridDim.x, blockIdx.x, vec4);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// The same sums accumulated in plain FP32 at every level (the "plain FP32"
// form the FP64-accurate reductions are compared against): per-thread sums,
// block sums and the final sum in FP32; the result is stored as a double.
template <int MODE>
__global__ void __launch_bounds__(kRT)
k_partial_fp32(const float* __restrict__ a, const float* __restrict__ b, long long n,
               double* __restrict__ partial) {
  pdl_enter();
  float acc = 0.f;
  const long long stride = (long long)gridDim.x * kRT;
  for (long long i = (long long)blockIdx.x * kRT + threadIdx.x; i < n; i += stride) {
    const float x = __ldg(a + i), y = __ldg(b + i);
    acc = MODE == 0 ? fmaf(x, y, acc) : fmaf(x - y, x - y, acc);
  }
  const float s = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = (double)s;
}

__global__ void __launch_bounds__(kRT)
k_final_sum_fp32(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  pdl_enter();
  float acc = 0.f;
  for (int i = threadIdx.x; i < nb; i += kRT) acc += (float)partial[i];
  const float s = block_sum(acc);
  if (threadIdx.x == 0) *out = (double)s;
}

__device__ __forceinline__ double final_sum(const double* __restrict__ partial, int nb) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += kRT) acc += partial[i];
  return block_sum(acc);
}

__global__ void __launch_bounds__(kRT)
k_final_sum(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  pdl_enter();
  const double s = final_sum(partial, nb);
  if (threadIdx.x == 0) *out = s;
}

static int aligned16(const void* a, const void* b) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u) == 0;
}

template <int MODE>
static void launch_sum(const float* a, const float* b, long long n, double* partial, double* out,
                       cudaStream_t st) {
  const int nb = reduce_blocks(n);
  if (t_plain_fp32_reduce) {
    launch_k(k_partial_fp32<MODE>, dim3(nb), dim3(kRT), 0, st, a, b, n, partial);
    launch_k(k_final_sum_fp32, dim3(1), dim3(kRT), 0, st, partial, nb, out);
    return;
  }
  launch_k(k_partial<MODE>, dim3(nb), dim3(kRT), 0, st, a, b, n, partial, aligned16(a, b));
  launch_k(k_final_sum, dim3(1), dim3(kRT), 0, st, partial, nb, out);
}

void launch_dot(const float* a, const float* b, long long n, double* partial, double* out,
                cudaStream_t st) {
  launch_sum<0>(a, b, n, partial, out, st);
}

void launch_sumsq_diff(const float* a, const float* b, long long n, double* partial,
                       double* out, cudaStream_t st) {
  launch_sum<1>(a, b, n, partial, out, st);
}

// block `bi` of `nblk`: the largest |a_i| (NaN propagates), valid in thread 0
__device__ __forceinline__ float partial_maxabs(const float* __restrict__ a, long long n, int nblk,
                                                int bi) {
  float m = 0.f;
  const long long stride = (long long)nblk * kRT;
#pragma unroll 4
  for (long long i = (long long)bi * kRT + threadIdx.x; i < n; i += stride) {
    const float x = fabsf(__ldg(a + i));
    m = (x > m || x != x) ? x : m;  // NaN propagates
  }
  __shared__ float ws[kRT / 32];
  m = warp_max(m);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = m;
  __syncthreads();
  float r = ws[0];
  if (threadIdx.x == 0)
    for (int k = 1; k < kRT / 32; ++k) r = (ws[k] > r || ws[k] != ws[k]) ? ws[k] : r;
  return r;
}

// the larger of two values, NaN if either is NaN
__device__ __forceinline__ float max_nan(float a, float b) { return (b > a || b != b) ? b : a; }

// the largest of nb partials by one warp (lane-strided, then across lanes;
// the maximum does not depend on the order), valid in every lane
__device__ __forceinline__ double final_maxabs(const float* __restrict__ partial, int nb) {
  const int lane = threadIdx.x & 31;
  float r = 0.f;
  for (int i = lane; i < nb; i += 32) r = max_nan(r, partial[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r = max_nan(r, __shfl_xor_sync(0xffffffffu, r, o));
  return (double)r;
}

__global__ void __launch_bounds__(kRT)
k_maxabs_partial(const float* __restrict__ a, long long n, float* __restrict__ partial) {
  pdl_enter();
  const float r = partial_maxabs(a, n, gridDim.x, blockIdx.x);
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void k_maxabs_final(const float* __restrict__ partial, int nb, double* out) {
  pdl_enter();
  const double r = final_maxabs(partial, nb);
  if (threadIdx.x == 0) *out = r;
}

void launch_maxabs(const float* a, long long n, float* partial, double* out, cudaStream_t st) {
  const int nb = reduce_blocks(n);
  launch_k(k_maxabs_partial, dim3(nb), dim3(kRT), 0, st, a, n, partial);
  launch_k(k_maxabs_final, dim3(1), dim3(32), 0, st, partial, nb, out);
}

// flag = 1 if any bit pattern differs (flag must be zeroed by the caller).
__global__ void k_compare(const unsigned* __restrict__ a, const unsigned* __restrict__ b,
                          long long n, int* flag) {
  pdl_enter();
  const long long stride = (long long)gridDim.x * blockDim.x;
  int d = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    d |= (__ldg(a + i) != __ldg(b + i));
  if (__syncthreads_or(d) && threadIdx.x == 0) atomicOr(flag, 1);
}

void launch_compare(const float* a, const float* b, long long n, int* flag, cudaStream_t st) {
  launch_k(k_compare, dim3(nblocks(n)), dim3(kRT), 0, st, reinterpret_cast<const unsigned*>(a),
           reinterpret_cast<const unsigned*>(b), n, flag);
}

__device__ __forceinline__ float lincomb_elem(float a, const float* x, float b, const float* y,
                                              long long i) {
  return y ? fmaf(b, y[i], a * x[i]) : a * x[i];
}

// z may alias x or y (elementwise, same index)
__global__ void k_lincomb(long long n, float a, const float* x, float b, const float* y,
                          float* z) {
  pdl_enter();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    z[i] = lincomb_elem(a, x, b, y, i);
}

void launch_lincomb(long long n, float a, const float* x, float b, const float* y, float* z,
                    cudaStream_t st) {
  launch_k(k_lincomb, dim3(nblocks(n)), dim3(kRT), 0, st, n, a, x, b, y, z);
}

// PCG step: alpha = rz / pq; x += alpha p; r -= alpha q. Nothing is changed
// when pq <= 0 (negative curvature: the host stops with x as it is).
__global__ void k_pcg_update(long long n, const double* rz, const double* pq,
                             const float* __restrict__ p, const float* __restrict__ q,
                             float* __restrict__ x, float* __restrict__ r) {
  pdl_enter();
  if (!(*pq > 0.0)) return;
  const double ad = *rz / *pq;
  const float alpha = (float)ad;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    x[i] = fmaf(alpha, p[i], x[i]);
    r[i] = fmaf(-alpha, q[i], r[i]);
  }
}

void launch_pcg_update(long long n, const double* rz, const double* pq, const float* p,
                       const float* q, float* x, float* r, cudaStream_t st) {
  launch_k(k_pcg_update, dim3(nblocks(n)), dim3(kRT), 0, st, n, rz, pq, p, q, x, r);
}

// p = z + (rz_new / rz_old) p
__global__ void k_pcg_direction(long long n, const double* rz_new, const double* rz_old,
                                const float* __restrict__ z, float* __restrict__ p) {
  pdl_enter();
  const float beta = (float)(*rz_new / *rz_old);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    p[i] = fmaf(beta, p[i], z[i]);
}

void launch_pcg_direction(long long n, const double* rz_new, const double* rz_old,
                          const float* z, float* p, cudaStream_t st) {
  launch_k(k_pcg_direction, dim3(nblocks(n)), dim3(kRT), 0, st, n, rz_new, rz_old, z, p);
}

__global__ void k_fill(float* x, long long n, float value) {
  pdl_enter();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    x[i] = value;
}

void launch_fill(float* x, long long n, float value, cudaStream_t st) {
  launch_k(k_fill, dim3(nblocks(n)), dim3(kRT), 0, st, x, n, value);
}

// SplitMix64 (Steele, Lea & Flood 2014): x[i] = uniform [-1, 1) from the
// (i+1)-th output of the stream started at seed.
__global__ void k_splitmix(float* x, long long n, unsigned long long seed) {
  pdl_enter();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    x[i] = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
  }
}

void launch_splitmix(float* x, long long n, unsigned long long seed, cudaStream_t st) {
  launch_k(k_splitmix, dim3(nblocks(n)), dim3(kRT), 0, st, x, n, seed);
}

// ---------------------------------------------------------------------------
// Batched forms (one launch over every problem of a batch, see SegView and
// BatchView): each problem's sums use its own partition and the device
// functions above, so every per-problem result is bitwise that of the
// one-problem reduction.

__device__ __forceinline__ const float* bref_c(const BRef& r, const BDesc& D) {
  return r.base + (long long)r.F * D.off + (long long)r.k * D.n1 * D.n2;
}

template <int MODE>
__global__ void __launch_bounds__(kRT)
k_partial_b(const BDesc* __restrict__ desc, SegView S, const int* __restrict__ mask, BRef a,
            BRef b, int L, double* __restrict__ partial) {
  pdl_enter();
  const int2 sb = S.blocks[blockIdx.x];
  if (!mask[sb.x]) return;
  const BDesc D = desc[sb.x];
  const float* pa = bref_c(a, D);
  const float* pb = bref_c(b, D);
  const int vec4 = ((reinterpret_cast<uintptr_t>(pa) | reinterpret_cast<uintptr_t>(pb)) & 15u) == 0;
  const double s = partial_sum<MODE>(pa, pb, (long long)L * D.n1 * D.n2, S.nb[sb.x], sb.y, vec4);
  if (threadIdx.x == 0) partial[S.first[sb.x] + sb.y] = s;
}

__global__ void __launch_bounds__(kRT)
k_final_sum_b(SegView S, const int* __restrict__ mask, const double* __restrict__ partial,
              double* __restrict__ out) {
  pdl_enter();
  const int p = blockIdx.x;
  if (!mask[p]) return;
  const double s = final_sum(partial + S.first[p], S.nb[p]);
  if (threadIdx.x == 0) out[p] = s;
}

__global__ void __launch_bounds__(kRT)
k_maxabs_partial_b(const BDesc* __restrict__ desc, SegView S, const int* __restrict__ mask,
                   BRef a, int L, float* __restrict__ partial) {
  pdl_enter();
  const int2 sb = S.blocks[blockIdx.x];
  if (!mask[sb.x]) return;
  const BDesc D = desc[sb.x];
  const float r = partial_maxabs(bref_c(a, D), (long long)L * D.n1 * D.n2, S.nb[sb.x], sb.y);
  if (threadIdx.x == 0) partial[S.first[sb.x] + sb.y] = r;
}

// one warp per problem
__global__ void k_maxabs_final_b(int nprob, SegView S, const int* __restrict__ mask,
                                 const float* __restrict__ partial, double* __restrict__ out) {
  pdl_enter();
  const int p = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (p >= nprob || !mask[p]) return;
  const double r = final_maxabs(partial + S.first[p], S.nb[p]);
  if ((threadIdx.x & 31) == 0) out[p] = r;
}

template <int MODE>
static void launch_sum_b(const BDesc* desc, const SegView& S, int nprob, const int* mask, BRef a,
                         BRef b, int L, double* partial, double* out, cudaStream_t st) {
  launch_k(k_partial_b<MODE>, dim3(S.nblocks), dim3(kRT), 0, st, desc, S, mask, a, b, L, partial);
  launch_k(k_final_sum_b, dim3(nprob), dim3(kRT), 0, st, S, mask, partial, out);
}

void launch_dot_b(const BDesc* desc, const SegView& S, int nprob, const int* mask, BRef a, BRef b,
                  int L, double* partial, double* out, cudaStream_t st) {
  launch_sum_b<0>(desc, S, nprob, mask, a, b, L, partial, out, st);
}

void launch_sumsq_diff_b(const BDesc* desc, const SegView& S, int nprob, const int* mask, BRef a,
                         BRef b, int L, double* partial, double* out, cudaStream_t st) {
  launch_sum_b<1>(desc, S, nprob, mask, a, b, L, partial, out, st);
}

void launch_maxabs_b(const BDesc* desc, const SegView& S, int nprob, const int* mask, BRef a,
                     int L, float* partial, double* out, cudaStream_t st) {
  launch_k(k_maxabs_partial_b, dim3(S.nblocks), dim3(kRT), 0, st, desc, S, mask, a, L, partial);
  launch_k(k_maxabs_final_b, dim3((nprob + 3) / 4), dim3(128), 0, st, nprob, S, mask, partial, out);
}

// problem of element e of an array of F fields per problem
__device__ __forceinline__ int elem_problem(const int* __restrict__ pmap, int F, long long e) {
  return pmap[(F == 1 ? e : e >> 1) >> 10];
}

__global__ void k_lincomb_b(const int* __restrict__ pmap, const int* __restrict__ mask, int F,
                            long long n, const float* __restrict__ a, const float* x,
                            const float* __restrict__ b, const float* y, float* z) {
  pdl_enter();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int p = elem_problem(pmap, F, i);
    if (mask[p]) z[i] = lincomb_elem(a[p], x, b ? b[p] : 0.f, y, i);
  }
}

void launch_lincomb_b(const int* pmap, const int* mask, int F, long long n, const float* a,
                      const float* x, const float* b, const float* y, float* z, cudaStream_t st) {
  launch_k(k_lincomb_b, dim3(nblocks(n)), dim3(kRT), 0, st, pmap, mask, F, n, a, x, b, y, z);
}

// Per-problem coefficients of the batched PCG updates, computed once per
// problem (FP64 divisions stay off the per-element path): the step
// alpha_p = (float)(rz_p / pq_p), on_p = 0 where the problem is masked or
// pq_p <= 0 (mode 0); the direction weight beta_p = (float)(rz_new_p /
// rz_old_p) (mode 1). The same roundings as the one-problem kernels.
__global__ void k_pcg_coef_b(int nprob, const int* __restrict__ mask, int mode,
                             const double* __restrict__ num, const double* __restrict__ den,
                             float* __restrict__ coef, int* __restrict__ on) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  const bool use = mask[p] && (mode == 1 || den[p] > 0.0);
  on[p] = use;
  coef[p] = use ? (float)(num[p] / den[p]) : 0.f;
}

__global__ void k_pcg_update_b(const int* __restrict__ pmap, int F, long long n,
                               const float* __restrict__ coef, const int* __restrict__ on,
                               const float* __restrict__ p, const float* __restrict__ q,
                               float* __restrict__ x, float* __restrict__ r) {
  pdl_enter();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int k = elem_problem(pmap, F, i);
    if (!on[k]) continue;
    const float alpha = coef[k];
    x[i] = fmaf(alpha, p[i], x[i]);
    r[i] = fmaf(-alpha, q[i], r[i]);
  }
}

void launch_pcg_update_b(const int* pmap, const int* mask, int nprob, int F, long long n,
                         const double* rz, const double* pq, float* coef, int* on, const float* p,
                         const float* q, float* x, float* r, cudaStream_t st) {
  launch_k(k_pcg_coef_b, dim3((nprob + 127) / 128), dim3(128), 0, st, nprob, mask, 0, rz, pq, coef, on);
  launch_k(k_pcg_update_b, dim3(nblocks(n)), dim3(kRT), 0, st, pmap, F, n, (const float*)coef,
           (const int*)on, p, q, x, r);
}

__global__ void k_pcg_direction_b(const int* __restrict__ pmap, int F, long long n,
                                  const float* __restrict__ coef, const int* __restrict__ on,
                                  const float* __restrict__ z, float* __restrict__ p) {
  pdl_enter();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int k = elem_problem(pmap, F, i);
    if (!on[k]) continue;
    p[i] = fmaf(coef[k], p[i], z[i]);
  }
}

void launch_pcg_direction_b(const int* pmap, const int* mask, int nprob, int F, long long n,
                            const double* rz_new, const double* rz_old, float* coef, int* on,
                            const float* z, float* p, cudaStream_t st) {
  launch_k(k_pcg_coef_b, dim3((nprob + 127) / 128), dim3(128), 0, st, nprob, mask, 1, rz_new, rz_old,
           coef, on);
  launch_k(k_pcg_direction_b, dim3(nblocks(n)), dim3(kRT), 0, st, pmap, F, n, (const float*)coef,
           (const int*)on, z, p);
}

__global__ void k_copy_scalars_b(int nprob, const int* __restrict__ mask,
                                 const double* __restrict__ src, double* __restrict__ dst) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nprob && mask[p]) dst[p] = src[p];
}

void launch_copy_scalars_b(int nprob, const int* mask, const double* src, double* dst,
                           cudaStream_t st) {
  launch_k(k_copy_scalars_b, dim3((nprob + 127) / 128), dim3(128), 0, st, nprob, mask, src, dst);
}

}  // namespace regnk
