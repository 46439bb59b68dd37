// Gauss-Newton data term of the Hessian matvec in one launch, synchronised
// tile by tile instead of step by step:
//     b~ = int_0^1 lambda~ grad m dt
// for a direction v~ (eq. hessian-matvec with every lambda term dropped,
// §3.4.1 footnote): the incremental state solve forward in time
// (eq. inc-state-slm) and the Gauss-Newton incremental adjoint solve backward
// (eq. inc-adj-slm without div(lambda v~)), cubic Lagrange interpolation
// (§3.5; the model of the two-level preconditioner's coarse problem), with the
// arithmetic of the per-step kernels k_incstate_step and k_adjoint_step of
// transport.cu, point for point.
//
// Why: on a grid whose points fit the GPU in one wave (the 512^2 coarse grid
// of P_2L: 262 144 points), a per-step kernel is a single dependent chain
// (displacement -> 4x4 gather -> store) whose duration is mostly launch and
// memory latency, and a matvec is 2 nt of them in a row. Here every block
// owns one 32 x 16 tile for the whole matvec. Step s of the 2 nt steps of a
// tile only reads the previous step's field within the reach of its stencils
// (ceil(max |displacement|) + 2 cells, i.e. the neighbouring tiles), so a
// block waits for those tiles' step s - 1 flags, not for the whole grid. The
// per-velocity fields of the tile (the two departure displacements, v~,
// v~(X_D), div v, div v at Y_D) and the running sum b~ stay in registers for
// all steps; per step only the time-level fields move (G_j and grad m_j
// forward, grad m_j backward) and the transported field is written once and
// gathered once: the algorithmic bytes of the matvec.
//
// Flags: one unsigned per tile, zeroed before the launch; a block publishes
// step s after all its stores (block barrier, fence, release store) and a
// waiting block polls its neighbours with relaxed loads, then takes one
// acquire fence. Two field buffers
// suffice: a tile starts step s only after its neighbours finished step
// s - 1, so nobody still reads the buffer it overwrites (step s - 2), and no
// neighbour can run ahead to step s + 1 before this tile has published s.
// Every block must be resident (cooperative launch, grid = tiles). A wait
// gives up after a bounded number of polls (~0.5 s), sets the error flag
// and the block returns; the other blocks then give up too and the host
// reports REG_ETIMEOUT.
#include "common.cuh"
#include "interp.cuh"
#include "kernels.h"

namespace regnk {

constexpr int kFlowTX = 32;                 // tile width (points)
constexpr int kFlowTY = 16;                 // tile height
constexpr int kFlowSP = 2;                  // adjacent points per thread
constexpr int kFlowT = kFlowTX * kFlowTY / kFlowSP;   // 256 threads
constexpr long long kFlowSpinLimit = 1LL << 21;

// polls read the flags with relaxed loads (no ordering, no L1 invalidation
// per poll); one acquire fence after the last successful poll orders the
// block's later loads after the neighbours' release stores
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int K>
__device__ __forceinline__ void fl_ld(const float* p, float (&a)[K]) {
  static_assert(K == 2, "two points per thread");
  const float2 t = __ldg(reinterpret_cast<const float2*>(p));
  a[0] = t.x;
  a[1] = t.y;
}

template <int K>
__device__ __forceinline__ void fl_st(float* p, const float (&a)[K]) {
  *reinterpret_cast<float2*>(p) = make_float2(a[0], a[1]);
}

// Tiles whose previous step this tile's stencils can reach: rx, ry tiles on
// each side (all tiles of an axis when 2 r + 1 covers it).
struct Reach {
  int x0, nx, y0, ny;
};

__device__ __forceinline__ Reach flow_reach(const FlowArgs& a, int tx, int ty) {
  const double d = fmax(a.dmax[0], a.dmax[1]);
  // a stencil at displacement d touches nodes floor(d) - 1 .. floor(d) + 2
  const double cells = (d >= 0.0 && d < 1e6) ? ceil(d) + 2.0 : 1e9;
  Reach r;
  const int rx = (int)fmin(ceil(cells / kFlowTX), 1e6), ry = (int)fmin(ceil(cells / kFlowTY), 1e6);
  if (2 * rx + 1 >= a.tiles_x) { r.x0 = 0; r.nx = a.tiles_x; } else { r.x0 = tx - rx; r.nx = 2 * rx + 1; }
  if (2 * ry + 1 >= a.tiles_y) { r.y0 = 0; r.ny = a.tiles_y; } else { r.y0 = ty - ry; r.ny = 2 * ry + 1; }
  return r;
}

// Waits until every tile in reach has published step s; false if a wait gave up.
__device__ __forceinline__ bool flow_wait(const FlowArgs& a, const Reach& r, int tile, unsigned s) {
  bool ok = true;
  const int K = r.nx * r.ny;
  // failure injection (tests): the first wait asks for a step nobody publishes
  const unsigned target = (a.inject && s == 1u) ? 0xFFFFFFFFu : s;
  for (int q = threadIdx.x; q < K && ok; q += kFlowT) {
    int nx = r.x0 + q % r.nx, ny = r.y0 + q / r.nx;
    nx = nx < 0 ? nx + a.tiles_x : (nx >= a.tiles_x ? nx - a.tiles_x : nx);
    ny = ny < 0 ? ny + a.tiles_y : (ny >= a.tiles_y ? ny - a.tiles_y : ny);
    const int nb = ny * a.tiles_x + nx;
    if (nb == tile) continue;
    const unsigned* f = a.flags + nb;
    long long spins = 0;
    while (ld_relaxed_u32(f) < target) {
      if (++spins > kFlowSpinLimit || *(volatile int*)a.err) {
        atomicExch(a.err, 1);
        ok = false;
        break;
      }
      __nanosleep(32);
    }
  }
  if (threadIdx.x < K) fence_acq_rel_gpu();
  return __syncthreads_or(!ok) == 0;
}

__device__ __forceinline__ void flow_publish(const FlowArgs& a, int tile, unsigned s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release_u32(a.flags + tile, s);
  }
}

// coherent gathers of the field written inside this launch (never the
// read-only path: the acquire of the neighbours' flags makes their stores
// visible to ordinary loads)
template <bool P2>
__device__ __forceinline__ float flow_gather(int i, int j, float d1, float d2, const FlowArgs& a,
                                             const float* src) {
  return apply_stencil<true>(make_stencil<P2>(i, j, d1, d2, a.n1, a.n2, a.log1, true), src);
}

template <bool P2>
__global__ void __launch_bounds__(kFlowT, 4) k_gn_flow(FlowArgs a) {
  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int t = threadIdx.x;
  constexpr int TPR = kFlowTX / kFlowSP;   // threads per tile row
  const int i0 = tx * kFlowTX + (t % TPR) * kFlowSP, j0 = ty * kFlowTY + t / TPR;
  const long long N = a.N;
  const long long idx = row_offset<P2>(j0, a.n1, a.log1) + i0;
  const float ht = a.ht, hh = 0.5f * ht;
  const int nt = a.nt;
  const Reach reach = flow_reach(a, tx, ty);

  // ---- incremental state, j = 1: v~(X_D) (kept) and m~_1 (m~_0 = 0)
  float x1[kFlowSP], x2[kFlowSP], u1[kFlowSP], u2[kFlowSP], w1[kFlowSP], w2[kFlowSP];
  float G1[kFlowSP], G2[kFlowSP], g1[kFlowSP], g2[kFlowSP], m[kFlowSP];
  fl_ld(a.dX + idx, x1);
  fl_ld(a.dX + N + idx, x2);
  fl_ld(a.vt + idx, u1);
  fl_ld(a.vt + N + idx, u2);
  fl_ld(a.G + idx, G1);
  fl_ld(a.G + N + idx, G2);
  fl_ld(a.gm + 2 * N + idx, g1);
  fl_ld(a.gm + 3 * N + idx, g2);
#pragma unroll
  for (int p = 0; p < kFlowSP; ++p) {
    const Stencil S = make_stencil<P2>(i0 + p, j0, x1[p], x2[p], a.n1, a.n2, a.log1, true);
    m[p] = 0.f;
    w1[p] = apply_stencil(S, a.vt);
    w2[p] = apply_stencil(S, a.vt + N);
  }
#pragma unroll
  for (int p = 0; p < kFlowSP; ++p)
    m[p] -= 0.5f * ht * (w1[p] * G1[p] + w2[p] * G2[p] + u1[p] * g1[p] + u2[p] * g2[p]);
  fl_st(a.buf1 + idx, m);
  flow_publish(a, tile, 1u);

  // ---- incremental state, j = 2..nt; the last one writes lambda~_nt =
  // -m~_nt and starts b~ = h_t/2 lambda~_nt grad m_nt
  // (m~_j = m~_{j-1}(X_D) - h_t/2 (v~(X_D) . G_j + v~ . grad m_j); the
  // operands of step s are requested before waiting for its neighbours)
  auto inc_step = [&](int s) -> bool {
    fl_ld(a.G + 2 * (long long)(s - 1) * N + idx, G1);
    fl_ld(a.G + (2 * (long long)(s - 1) + 1) * N + idx, G2);
    fl_ld(a.gm + 2 * (long long)s * N + idx, g1);
    fl_ld(a.gm + (2 * (long long)s + 1) * N + idx, g2);
    if (!flow_wait(a, reach, tile, (unsigned)(s - 1))) return false;
    const float* src = (s & 1) ? a.buf0 : a.buf1;   // step s - 1
#pragma unroll
    for (int p = 0; p < kFlowSP; ++p) m[p] = flow_gather<P2>(i0 + p, j0, x1[p], x2[p], a, src);
#pragma unroll
    for (int p = 0; p < kFlowSP; ++p)
      m[p] -= 0.5f * ht * (w1[p] * G1[p] + w2[p] * G2[p] + u1[p] * g1[p] + u2[p] * g2[p]);
    return true;
  };
  for (int s = 2; s < nt; ++s) {
    if (!inc_step(s)) return;
    fl_st(((s & 1) ? a.buf1 : a.buf0) + idx, m);
    flow_publish(a, tile, (unsigned)s);
  }
  if (!inc_step(nt)) return;
  float b1[kFlowSP], b2[kFlowSP];
#pragma unroll
  for (int p = 0; p < kFlowSP; ++p) {
    m[p] = -m[p];
    b1[p] = hh * m[p] * g1[p];
    b2[p] = hh * m[p] * g2[p];
  }
  fl_st(((nt & 1) ? a.buf1 : a.buf0) + idx, m);
  flow_publish(a, tile, (unsigned)nt);

  // ---- Gauss-Newton incremental adjoint, j = nt-1..0 (step s = 2 nt - j)
  float y1[kFlowSP], y2[kFlowSP], dd[kFlowSP], db[kFlowSP], l[kFlowSP];
  fl_ld(a.dY + idx, y1);
  fl_ld(a.dY + N + idx, y2);
  fl_ld(a.delta + idx, dd);
  fl_ld(a.delta_bar + idx, db);
  for (int s = nt + 1; s <= 2 * nt; ++s) {
    const int jt = 2 * nt - s;
    const float wb = ht * (jt == 0 ? 0.5f : 1.0f);
    fl_ld(a.gm + 2 * (long long)jt * N + idx, g1);
    fl_ld(a.gm + (2 * (long long)jt + 1) * N + idx, g2);
    if (!flow_wait(a, reach, tile, (unsigned)(s - 1))) return;
    const float* src = (s & 1) ? a.buf0 : a.buf1;   // step s - 1
#pragma unroll
    for (int p = 0; p < kFlowSP; ++p) l[p] = flow_gather<P2>(i0 + p, j0, y1[p], y2[p], a, src);
#pragma unroll
    for (int p = 0; p < kFlowSP; ++p) {
      const float lstar = fmaf(ht * l[p], db[p], l[p]);
      l[p] = l[p] + 0.5f * ht * (l[p] * db[p] + lstar * dd[p]);
    }
#pragma unroll
    for (int p = 0; p < kFlowSP; ++p) {
      b1[p] = fmaf(wb * l[p], g1[p], b1[p]);
      b2[p] = fmaf(wb * l[p], g2[p], b2[p]);
    }
    if (s < 2 * nt) {   // lambda~_0 is only needed for b~
      fl_st(((s & 1) ? a.buf1 : a.buf0) + idx, l);
      flow_publish(a, tile, (unsigned)s);
    }
  }
  fl_st(a.b + idx, b1);
  fl_st(a.b + N + idx, b2);
}

static bool flow_pow2(int n1, int n2) { return !(n1 & (n1 - 1)) && !(n2 & (n2 - 1)); }

int flow_tiles(int n1, int n2) {
  if (n1 % kFlowTX || n2 % kFlowTY) return 0;
  return (n1 / kFlowTX) * (n2 / kFlowTY);
}

// resident blocks of k_gn_flow on the current device (0 if unknown)
int flow_capacity(int n1, int n2) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const auto k = flow_pow2(n1, n2) ? k_gn_flow<true> : k_gn_flow<false>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kFlowT, 0) != cudaSuccess) return 0;
  return sms * per;
}

cudaError_t launch_gn_flow(const FlowArgs& a, cudaStream_t st) {
  const int tiles = a.tiles_x * a.tiles_y;
  cudaError_t e = cudaMemsetAsync(a.flags, 0, (size_t)tiles * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles);
  cfg.blockDim = dim3(kFlowT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, flow_pow2(a.n1, a.n2) ? k_gn_flow<true> : k_gn_flow<false>, a);
  ++g_launch_count;
  return e;
}

}  // namespace regnk
