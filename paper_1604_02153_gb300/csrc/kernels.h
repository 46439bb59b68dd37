// Internal launch interface between the kernels and the host runtime.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <utility>

#include "interp.cuh"

namespace regnk {

// Kernel launches issued by the library since load (incremented after every
// launch, from any host thread; read by reg_launch_count).
extern std::atomic<long long> g_launch_count;

// Programmatic dependent launch. A kernel launched through launch_k carries
// the programmatic-stream-serialisation attribute: the GPU may schedule its
// blocks while the preceding kernel of the stream is still running, which
// hides the launch latency between the many short dependent kernels of a
// transport sweep. Every kernel launched this way calls pdl_enter() before
// its first global memory access: griddepcontrol.wait blocks until the
// preceding kernel has completed and its writes are visible (it returns at
// once for a kernel launched without the attribute), and only then does the
// kernel allow its own successor to be scheduled. No data is read early, so
// the results do not depend on the attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Attribute value for launches from this host thread (reg_options
// .programmatic_launch of the context being driven; 1 outside a context).
extern thread_local int t_programmatic_launch;
// While a CUDA graph is captured: 1 = launches on the coarse grid level carry
// the attribute as well, 2 = all launches do (reg_options.graph_pdl); the
// level of the launches being issued (0 problem grid, 1 coarse grid).
extern thread_local int t_graph_pdl;
extern thread_local int t_level;
// 1 while a context with reg_options.precision = REG_PRECISION_FP32 runs a
// call: inner products and squared norms accumulate in plain FP32
extern thread_local int t_plain_fp32_reduce;

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed =
      (t_programmatic_launch || t_graph_pdl == 2 || (t_graph_pdl == 1 && t_level == 1)) ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  ++g_launch_count;
}

// Spectral multipliers of the column pass (see fft.cu).
enum SpecOp {
  SPOP_SCALE = 0,        // sigma = 1 (with resampling: restriction / prolongation)
  SPOP_GRAD = 1,         // 1 -> 2: i k1, i k2 (Nyquist zeroed)
  SPOP_DIV = 2,          // 2 -> 1: i k1 u1 + i k2 u2 (Nyquist zeroed)
  SPOP_REGPOW = 3,       // (beta |k|^2p)^s, s = 1 exact, otherwise k = 0 weight -> 1
  SPOP_LOWPASS = 4,      // |k1| < n1/4 and |k2| < n2/4
  SPOP_HIGHPASS = 5,     // complement of LOWPASS
  SPOP_REGPOW_HIGH = 6,  // REGPOW restricted to the high band
  SPOP_LERAY = 7,        // 2 -> 2: delta_oc - k_o k_c / |k|^2 (Nyquist zeroed; 1 where |k| = 0)
  SPOP_REGPOW_LERAY = 8, // 2 -> 2: REGPOW times LERAY
  SPOP_REGW = 9,         // 2 -> 2: R^s, R = beta A - beta_w grad (I - Lap) div (near-incompressible)
  SPOP_KW = 10,          // 2 -> 2: near-incompressible K = I - c(k) kd kd^T / |kd|^2
  SPOP_REGPOW_KW = 11,   // 2 -> 2: REGPOW times KW
};

// Optional skip of whole fields in one FFT launch (batches of problems): a
// block working on field (or group) u of the launch returns at once when
// mask[p0 + u / per] is zero. mask = NULL: every field is transformed.
struct FieldMask {
  const int* mask = nullptr;
  int p0 = 0;
  int per = 1;
};

struct ColArgs {
  const float2* in;
  long long in_fstride;   // complex values between consecutive input spectra
  float2* out;
  long long out_fstride;
  int nin, nout;          // spectra per group in and out
  int nk1_out;            // output lines (n1_out / 2 + 1)
  int n1_in, n2_in, n1_out, n2_out;
  int n1, n2;             // grid the Nyquist / filter conditions refer to
  int op;
  float beta;
  int p;
  float s;
  float beta_w;           // weight of the divergence norm (SPOP_REGW*)
  float scale;            // 1 / (n1_in n2_in)
  const float2* tw_in;    // twiddles for length n2_in
  const float2* tw_out;   // twiddles for length n2_out
  FieldMask fm;           // groups to skip (per = groups per problem)
};

// fft.cu
void fft_rows_r2c(int n1, int n2, const float* in, long long fstride, float2* spec,
                  long long sstride, int F, const float2* tw, cudaStream_t st,
                  const FieldMask& fm = FieldMask{});
// Optional epilogue of the inverse row pass: with Ad = the pass's output
// plus its addend, one Chebyshev iteration r -= Ad; d = a d + b r; x += d on
// the same points, instead of storing Ad. The addend, if any, must be d
// itself (the operator is applied to d); the vectors have the pass's field
// layout (field f at offset f * fstride).
struct ChebEpilogue {
  float* r = nullptr;
  float* d = nullptr;
  float* x = nullptr;
  float a = 0.f, b = 0.f;
};
void fft_rows_c2r(int n1, int n2, const float2* spec, long long sstride, float* out,
                  long long fstride, const float* add, long long astride, int F,
                  const float2* tw, cudaStream_t st,
                  const ChebEpilogue* cheb = nullptr, const FieldMask& fm = FieldMask{});
void fft_cols(const ColArgs& a, int groups, cudaStream_t st);
// n = 2^L (L = 5..11) or 3 * 2^L (L = 5..9)
bool fft_size_supported(int n);
// 3D grids: complex FFTs along one axis of F arrays of `total` values (see
// k_axis); n = 32, 64, 128, 256, 96 or 192
bool fft_axis_supported(int n);
void fft_axis(float2* z, long long total, int F, int n, long long inner, bool inverse,
              const float2* tw, cudaStream_t st);

// transport.cu
struct PrefilterTaps;  // host-computed, passed by value below
void launch_prefilter(int n1, int n2, const float* in, float* tmp, float* out, int F,
                      cudaStream_t st);
void launch_departure(int n1, int n2, float ht, const float* v, const float* cv,
                      float* dX, float* dY, int lagrange, cudaStream_t st);
void launch_gather(int n1, int n2, const float* coef, const float* disp, float* out, int F,
                   long long fstride, int lagrange, cudaStream_t st);
void launch_state_step(int n1, int n2, const float* coef, const float* dX, float* out,
                       int lagrange, cudaStream_t st);
void launch_adjoint_init(int n1, int n2, float coef_b, const float* mR, const float* m1,
                         const float* gm, float* lam, float* b, float sign, cudaStream_t st);
// Tile shapes of the step kernels (launch_adjoint_step, launch_incstate_step):
// index 1..kStepTiles, threads per block 128 << ((k - 1) / 3), points per
// thread 1 << ((k - 1) % 3).
constexpr int kStepTiles = 9;
constexpr int kDefaultStepTile = 5;   // 256 threads x 2 points
inline int step_tile_threads(int k) { return 128 << ((k - 1) / 3); }
inline int step_tile_points(int k) { return 1 << ((k - 1) % 3); }
void launch_adjoint_step(int tile, int n1, int n2, float ht, float wb, const float* coef,
                         const float* dY, const float* delta, const float* delta_bar,
                         const float* gm, float* lam_out, float* b, int lagrange,
                         cudaStream_t st);
// Full-Newton incremental adjoint (transport.cu): products lambda_j v~ of L
// time levels, the final condition with the first term of the time
// integral, and one backward step with the div(lambda v~) source.
void launch_lam_times_vt(long long N, int L, const float* lam, const float* vt, float* out,
                         cudaStream_t st);
void launch_fn_adjoint_init(long long N, float coef_b, const float* mt, const float* gm,
                            const float* lam, const float* gmt, float* lt, float* b,
                            cudaStream_t st);
void launch_fn_adjoint_step(int n1, int n2, float ht, float wb, const float* coef_l,
                            const float* coef_s, const float* dY, const float* delta,
                            const float* delta_bar, const float* src, const float* gm,
                            const float* lam, const float* gmt, float* lt_out, float* b,
                            int lagrange, cudaStream_t st);
// RK2A comparator: one Heun stage of the antisymmetric-form state (s = -1)
// or adjoint (s = +1) equation (transport.cu).
void launch_rk2a_stage(long long N, float s, const float* u, const float* g, const float* v,
                       const float* dv, const float* delta, const float* base, float a,
                       const float* kprev, float b, float* out, float* kout, cudaStream_t st);
// det grad y from the four spectral derivatives of u = y - x (transport.cu).
void launch_det_grad(long long N, const float* g, float* det, cudaStream_t st);
// Fused prefilter + step kernels (transport.cu). fused_box_width gives the
// box width (48 or 64) whose halo covers displacements up to max_disp_cells,
// or 0 if none does; fused_init raises the kernels' shared-memory limit
// (call once per device before the first launch).
int fused_box_width(double max_disp_cells);
void fused_init();
void launch_adjoint_fused(int W, int n1, int n2, float ht, float wb, const float* lam_next,
                          const float* dY, const float* delta, const float* delta_bar,
                          const float* gm, float* lam_out, float* b, cudaStream_t st);
void launch_incstate_fused(int W, int n1, int n2, float ht, const float* m_prev, const float* dX,
                           const float* vt, const float* vtD, const float* G, const float* gm,
                           float* out, const float* gm_nt, float* b, cudaStream_t st);
void launch_gather_fused(int W, int n1, int n2, const float* u, long long fstride, int F,
                         const float* disp, float* out, cudaStream_t st);
void launch_incstate_first_fused(int W, int n1, int n2, float ht, const float* vt, const float* dX,
                                 const float* G1, const float* gm1, float* vtD, float* out,
                                 cudaStream_t st);
void launch_incstate_step(int tile, int n1, int n2, float ht, const float* coef, const float* dX,
                          const float* vt, float* vtD, const float* G, const float* gm,
                          float* out, int first, int lagrange, cudaStream_t st,
                          const float* cvt = nullptr, const float* gm_nt = nullptr,
                          float* b = nullptr);

// matvec.cu: persistent Gauss-Newton data-term matvec (one cooperative launch)
struct MatvecArgs {
  int n1, n2, log1, nt, lagrange;
  long long N;
  float ht;
  const float* vt;          // direction v~ (2N)
  const float* dX;          // forward departure displacement (2N)
  const float* dY;          // backward departure displacement (2N)
  const float* delta;       // div v (N)
  const float* delta_bar;   // div v at Y_D (N)
  const float* gm;          // grad m_0..grad m_nt (2 (nt+1) N)
  const float* G;           // grad m_{j-1}(X_D), j = 1..nt (2 nt N)
  float* c2;                // scratch: coefficients of v~ (2N)
  float* vtD;               // scratch: v~(X_D) (2N)
  float* fA;                // scratch (N)
  float* fB;                // scratch (N)
  float* coef;              // scratch: coefficients of one field (N)
  float* b;                 // output: the data term b~ (2N)
  unsigned* bar;            // grid barrier: counter, generation (self-resetting)
  int* err;                 // set when a barrier wait gave up
  unsigned missing;         // failure injection: arrivals that never come (tests)
};
cudaError_t launch_gn_matvec(const MatvecArgs& a, cudaStream_t st);

// flow.cu: the GN data term in one launch with tile-to-tile synchronisation
// (cubic Lagrange model, nt >= 2, every tile's block resident)
struct FlowArgs {
  int n1, n2, log1, nt;
  long long N;
  float ht;
  int tiles_x, tiles_y;     // 32 x 16 point tiles
  const float* vt;          // direction v~ (2N)
  const float* dX;          // forward departure displacement (2N)
  const float* dY;          // backward departure displacement (2N)
  const float* delta;       // div v (N)
  const float* delta_bar;   // div v at Y_D (N)
  const float* gm;          // grad m_0..grad m_nt (2 (nt+1) N)
  const float* G;           // grad m_{j-1}(X_D), j = 1..nt (2 nt N)
  float* buf0;              // scratch: the transported field, two steps (N each)
  float* buf1;
  float* b;                 // output: the data term b~ (2N)
  unsigned* flags;          // one per tile (zeroed by launch_gn_flow)
  int* err;                 // set when a wait gave up
  const double* dmax;       // largest |displacement| of X_D and of Y_D in cells (device)
  int inject;               // failure injection (tests): 1 = the first wait never ends
};
int flow_tiles(int n1, int n2);
int flow_capacity(int n1, int n2);
cudaError_t launch_gn_flow(const FlowArgs& a, cudaStream_t st);

// reduce.cu
void launch_dot(const float* a, const float* b, long long n, double* partial, double* out,
                cudaStream_t st);
void launch_sumsq_diff(const float* a, const float* b, long long n, double* partial,
                       double* out, cudaStream_t st);
void launch_maxabs(const float* a, long long n, float* partial, double* out, cudaStream_t st);
void launch_compare(const float* a, const float* b, long long n, int* flag, cudaStream_t st);
void launch_lincomb(long long n, float a, const float* x, float b, const float* y, float* z,
                    cudaStream_t st);
void launch_pcg_update(long long n, const double* rz, const double* pq, const float* p,
                       const float* q, float* x, float* r, cudaStream_t st);
void launch_pcg_direction(long long n, const double* rz_new, const double* rz_old,
                          const float* z, float* p, cudaStream_t st);
void launch_fill(float* x, long long n, float value, cudaStream_t st);
void launch_splitmix(float* x, long long n, unsigned long long seed, cudaStream_t st);
int reduce_partials();
// Blocks (partial sums) of the two-stage reduction of n values: four float4
// per thread of a 256-thread block, at most reduce_partials(). The batched
// reductions use the same partition per problem, so both give the same bits.
inline int reduce_blocks(long long n) {
  const long long b = (n + 16LL * 256 - 1) / (16LL * 256);
  return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

// ---------------------------------------------------------------------------
// Batches of problems advanced in lockstep (lockstep.cu): one launch per
// transport step over the 32 x 32 tiles of every problem of the batch.
//
// Every array of a batch holds, for each problem p in order, a block of F
// grid-sized fields (F fixed per array: 1 for a scalar field, 2 for a vector
// field, nt + 1 for a state history, ...), so problem p's block starts at
// F * off_p with off_p the sum of the earlier problems' point counts, and its
// field k at F * off_p + k * N_p. A BRef names field k of such an array for
// every problem at once.
struct BDesc {
  int n1, n2;
  int log1;          // log2(n1) when both lengths are powers of two, else -1
  int p2;            // both lengths powers of two
  long long off;     // off_p (a multiple of 1024)
  float s1, s2;      // h_t n_i / (2 pi): velocity to cells per time step
};

struct BRef {
  float* base;       // NULL: no such field (an optional argument)
  int F;             // fields per problem in the array
  int k;             // field index within the problem's block
};

// What the batched kernels read about the batch. w and mask are written on
// the device (w, per velocity) and by the host (mask, per phase).
struct BatchView {
  const BDesc* desc;   // per problem
  const int* w;        // box width of the fused kernels (48 or 64; 0: a
                       // displacement beyond their halo: the problem's
                       // blocks skip the step)
  const int* mask;     // nonzero: the problem takes part in this phase
  const int4* tiles;   // per tile block: problem, tile column, tile row
  const int* pmap;     // per 1024 consecutive points of the batch: problem
  int ntiles;
};

// Per-problem partition of a reduction over L fields of each problem
// (L * N_p values), the same as the one-problem reduction of L * N_p
// values uses: nb[p] blocks whose partial sums sit at partial[first[p] ..].
struct SegView {
  const int2* blocks;  // per block: problem, block index within the problem
  const int* nb;       // per problem
  const int* first;    // per problem
  int nblocks;
};

// transport.cu
// h_t n / (2 pi) in FP32: a velocity in radians per unit time to cells per step
float departure_scale(float ht, int n);
void batch_fused_init();
void launch_prefilter_b(const BatchView& B, BRef in, BRef out, int F, cudaStream_t st);
void launch_departure_b(const BatchView& B, long long npts, BRef v, BRef cv, BRef dX, BRef dY,
                        cudaStream_t st);
void launch_copy_field_b(const BatchView& B, long long npts, BRef src, BRef dst, cudaStream_t st);
void launch_set_w_b(int nprob, const double* dmax_x, const double* dmax_y, int* w, cudaStream_t st);
void launch_adjoint_init_b(const BatchView& B, long long npts, float coef_b, BRef mR, BRef m1,
                           BRef gm, BRef lam, BRef b, float sign, cudaStream_t st);
void launch_gather_fused_b(const BatchView& B, BRef u, int F, BRef disp, BRef out,
                           cudaStream_t st);
void launch_adjoint_fused_b(const BatchView& B, float ht, float wb, BRef lam_next, BRef dY,
                            BRef delta, BRef delta_bar, BRef gm, BRef lam_out, BRef b,
                            cudaStream_t st);
void launch_incstate_first_fused_b(const BatchView& B, float ht, BRef vt, BRef dX, BRef G1,
                                   BRef gm1, BRef vtD, BRef out, cudaStream_t st);
void launch_incstate_fused_b(const BatchView& B, float ht, BRef m_prev, BRef dX, BRef vt,
                             BRef vtD, BRef G, BRef gm, BRef out, BRef gm_nt, BRef b,
                             cudaStream_t st);

// reduce.cu: per-problem sums (FP64 result per problem in out[p]) with the
// arithmetic and summation order of the one-problem reductions, masked
// problems skipped; per-problem Krylov updates.
void launch_dot_b(const BDesc* desc, const SegView& S, int nprob, const int* mask, BRef a, BRef b,
                  int L, double* partial, double* out, cudaStream_t st);
void launch_sumsq_diff_b(const BDesc* desc, const SegView& S, int nprob, const int* mask, BRef a,
                         BRef b, int L, double* partial, double* out, cudaStream_t st);
void launch_maxabs_b(const BDesc* desc, const SegView& S, int nprob, const int* mask, BRef a,
                     int L, float* partial, double* out, cudaStream_t st);
// z = a_p x + b_p y on the problems of the mask (arrays of F fields per
// problem, n = F * total points; a_p, b_p per problem; y may be NULL)
void launch_lincomb_b(const int* pmap, const int* mask, int F, long long n, const float* a,
                      const float* x, const float* b, const float* y, float* z, cudaStream_t st);
// (coef, on: per-problem scratch of nprob entries)
void launch_pcg_update_b(const int* pmap, const int* mask, int nprob, int F, long long n,
                         const double* rz, const double* pq, float* coef, int* on, const float* p,
                         const float* q, float* x, float* r, cudaStream_t st);
void launch_pcg_direction_b(const int* pmap, const int* mask, int nprob, int F, long long n,
                            const double* rz_new, const double* rz_old, float* coef, int* on,
                            const float* z, float* p, cudaStream_t st);
void launch_copy_scalars_b(int nprob, const int* mask, const double* src, double* dst,
                           cudaStream_t st);

}  // namespace regnk
