// Persistent Gauss-Newton data-term matvec: one cooperative launch computes
//     b~ = int_0^1 lambda~ grad m dt
// for a direction v~ (eq. hessian-matvec with every lambda term dropped,
// §3.4.1 footnote): the incremental state solve forward in time
// (eq. inc-state-slm) and the Gauss-Newton incremental adjoint solve backward
// (eq. inc-adj-slm without div(lambda v~)), with the same arithmetic as the
// per-step kernels of transport.cu.
//
// A multi-kernel matvec launches ~4 nt + 8 kernels; on small grids (the
// 512^2 coarse grid of the two-level preconditioner) each of them is too
// short to fill the GPU and launch latency dominates. Here the blocks stay
// resident and step through the phases, separated by a grid-wide barrier:
//     prefilter v~ | v~(X_D), m~_1 | (prefilter m~_{j-1} | m~_j) j = 2..nt |
//     (prefilter lambda~_{j+1} | lambda~_j, b~ += ...) j = nt-1..0
// (prefilter phases are absent for the Lagrange model). Data produced inside
// the kernel is read with ordinary loads, never through the read-only path:
// the barrier's release/acquire fences make them observe the other blocks'
// writes while still letting neighbouring stencils share L1 lines.
//
// The barrier is a counter plus a generation word in global memory. A block
// that waits longer than ~0.5 s (bounded spin with __nanosleep) sets the
// error flag and every block leaves at the next barrier; the host turns the
// flag into REG_ETIMEOUT. With a cooperative launch all blocks are resident,
// so the wait ends in normal operation.
#include "common.cuh"
#include "interp.cuh"
#include "kernels.h"

namespace regnk {

constexpr int kMT = kPThreads;           // threads per block (256)
constexpr long long kSpinLimit = 1LL << 23;

// `missing` > 0 makes the barrier wait for arrivals that never come (used by
// the failure-detection test: every block times out and the kernel ends).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned missing) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1 + missing) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (++spins > kSpinLimit || *(volatile int*)err) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err == 0;
}

template <bool LAGRANGE, bool P2>
__device__ __forceinline__ void prefilter_phase(const MatvecArgs& a, const float* src, float* dst,
                                                int F, float* sin_, float* smid) {
  if (LAGRANGE) return;
  const int tx = a.n1 / kPX, tiles = tx * (a.n2 / kPY);
  for (int w = blockIdx.x; w < F * tiles; w += gridDim.x) {
    const int f = w / tiles, tile = w - f * tiles;
    const int x0 = (tile % tx) * kPX, y0 = (tile / tx) * kPY;
    prefilter_tile<P2, true>(src + f * a.N, dst + f * a.N, a.n1, a.n2, a.log1, x0, y0, sin_, smid);
    __syncthreads();
  }
}

template <bool LAGRANGE, bool P2>
__global__ void __launch_bounds__(kMT) k_gn_matvec(MatvecArgs a) {
  __shared__ float sin_[kPH * kPIn];
  __shared__ float smid[kPH * kPMid];
  const long long N = a.N;
  const int n1 = a.n1, n2 = a.n2, log1 = a.log1, nt = a.nt;
  const float ht = a.ht, hh = 0.5f * ht;
  const long long stride = (long long)gridDim.x * kMT;
  const long long first = (long long)blockIdx.x * kMT + threadIdx.x;

  // phase: interpolation coefficients of v~
  const float* cvt = a.vt;
  if (!LAGRANGE) {
    prefilter_phase<LAGRANGE, P2>(a, a.vt, a.c2, 2, sin_, smid);
    cvt = a.c2;
    if (!grid_barrier(a.bar, a.err, a.missing)) return;
  }
  // phase: v~(X_D) and the first incremental state step (m~_0 = 0)
  float* cur = a.fA;
  float* nxt = a.fB;
  const float* gm_nt = a.gm + 2 * (long long)nt * N;
  for (long long idx = first; idx < N; idx += stride) {
    int i, j;
    split_index<P2>(idx, n1, log1, i, j);
    const Stencil S = make_stencil<P2>(i, j, __ldg(a.dX + idx), __ldg(a.dX + N + idx), n1, n2, log1,
                                   LAGRANGE);
    const float w1 = apply_stencil<true>(S, cvt), w2 = apply_stencil<true>(S, cvt + N);
    a.vtD[idx] = w1;
    a.vtD[N + idx] = w2;
    const float* G1 = a.G;
    const float* g1 = a.gm + 2 * N;
    const float src = w1 * __ldg(G1 + idx) + w2 * __ldg(G1 + N + idx) +
                      __ldg(a.vt + idx) * __ldg(g1 + idx) + __ldg(a.vt + N + idx) * __ldg(g1 + N + idx);
    const float m = -hh * src;
    if (nt == 1) {   // lambda~_1 = -m~_1 and the t = 1 term of the time integral
      cur[idx] = -m;
      a.b[idx] = hh * (-m) * __ldg(gm_nt + idx);
      a.b[N + idx] = hh * (-m) * __ldg(gm_nt + N + idx);
    } else {
      cur[idx] = m;
    }
  }
  if (!grid_barrier(a.bar, a.err, a.missing)) return;
  // incremental state, j = 2..nt
  for (int jt = 2; jt <= nt; ++jt) {
    const float* coef = cur;
    if (!LAGRANGE) {
      prefilter_phase<LAGRANGE, P2>(a, cur, a.coef, 1, sin_, smid);
      coef = a.coef;
      if (!grid_barrier(a.bar, a.err, a.missing)) return;
    }
    const float* Gj = a.G + 2 * (long long)(jt - 1) * N;
    const float* gj = a.gm + 2 * (long long)jt * N;
    for (long long idx = first; idx < N; idx += stride) {
      int i, j;
      split_index<P2>(idx, n1, log1, i, j);
      const Stencil S = make_stencil<P2>(i, j, __ldg(a.dX + idx), __ldg(a.dX + N + idx), n1, n2,
                                     log1, LAGRANGE);
      const float base = apply_stencil<true>(S, coef);
      const float src = __ldca(a.vtD + idx) * __ldg(Gj + idx) + __ldca(a.vtD + N + idx) * __ldg(Gj + N + idx) +
                        __ldg(a.vt + idx) * __ldg(gj + idx) + __ldg(a.vt + N + idx) * __ldg(gj + N + idx);
      const float m = base - hh * src;
      if (jt == nt) {   // lambda~_nt = -m~_nt (eq. inc-adj-fc-elim) and b~ init
        nxt[idx] = -m;
        a.b[idx] = hh * (-m) * __ldg(gm_nt + idx);
        a.b[N + idx] = hh * (-m) * __ldg(gm_nt + N + idx);
      } else {
        nxt[idx] = m;
      }
    }
    float* t = cur;
    cur = nxt;
    nxt = t;
    if (!grid_barrier(a.bar, a.err, a.missing)) return;
  }
  // Gauss-Newton incremental adjoint, j = nt-1..0, cur = lambda~_{j+1}
  for (int jt = nt - 1; jt >= 0; --jt) {
    const float* coef = cur;
    if (!LAGRANGE) {
      prefilter_phase<LAGRANGE, P2>(a, cur, a.coef, 1, sin_, smid);
      coef = a.coef;
      if (!grid_barrier(a.bar, a.err, a.missing)) return;
    }
    const float wb = ht * (jt == 0 ? 0.5f : 1.0f);
    const float* gj = a.gm + 2 * (long long)jt * N;
    for (long long idx = first; idx < N; idx += stride) {
      int i, j;
      split_index<P2>(idx, n1, log1, i, j);
      const Stencil S = make_stencil<P2>(i, j, __ldg(a.dY + idx), __ldg(a.dY + N + idx), n1, n2,
                                     log1, LAGRANGE);
      const float lb = apply_stencil<true>(S, coef);
      const float db = __ldg(a.delta_bar + idx), d = __ldg(a.delta + idx);
      const float lstar = fmaf(ht * lb, db, lb);
      const float l = lb + 0.5f * ht * (lb * db + lstar * d);
      nxt[idx] = l;
      a.b[idx] = fmaf(wb * l, __ldg(gj + idx), __ldca(a.b + idx));
      a.b[N + idx] = fmaf(wb * l, __ldg(gj + N + idx), __ldca(a.b + N + idx));
    }
    float* t = cur;
    cur = nxt;
    nxt = t;
    if (jt > 0 && !grid_barrier(a.bar, a.err, a.missing)) return;
  }
}

static bool pow2_args(const MatvecArgs& a) {
  return !(a.n1 & (a.n1 - 1)) && !(a.n2 & (a.n2 - 1));
}

// the four instantiations, indexed by 2 * lagrange + pow2
using MatvecKernel = void (*)(MatvecArgs);
static const MatvecKernel kMatvecKernels[4] = {k_gn_matvec<false, false>, k_gn_matvec<false, true>,
                                               k_gn_matvec<true, false>, k_gn_matvec<true, true>};

static std::atomic<int> g_matvec_blocks[4][64];

// resident blocks of a cooperative launch of variant k on the current device
static int matvec_grid(int k) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 0;
  std::atomic<int>& slot = g_matvec_blocks[k][dev];
  int nb = slot.load();
  if (nb == 0) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kMatvecKernels[k], kMT, 0);
    per = per > 2 ? 2 : per;   // two blocks per SM: enough threads, few barrier arrivals
    nb = sms * per;
    slot.store(nb);
  }
  return nb;
}

cudaError_t launch_gn_matvec(const MatvecArgs& a, cudaStream_t st) {
  const int k = 2 * (a.lagrange ? 1 : 0) + (pow2_args(a) ? 1 : 0);
  const int nb = matvec_grid(k);
  if (nb <= 0) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(kMT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kMatvecKernels[k], a);
  ++g_launch_count;
  return e;
}

}  // namespace regnk
