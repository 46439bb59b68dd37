// Many registration problems of uneven grid size advanced in lockstep.
//
// The problems share one set of device arrays: problem p's fields are one
// block of each array, described by a table of (n1, n2, offset) per problem
// (BDesc). Every semi-Lagrangian step (departure points, state, adjoint,
// incremental state and adjoint, the gathers of div v and of the gradient
// history) is ONE launch over the 32 x 32 tiles of every problem; every FFT
// pass is one launch per group of consecutive problems with the same grid and
// beta (the problems are ordered so that such groups are contiguous); each
// per-problem inner product or norm is one segmented reduction over all
// problems with an FP64 result per problem. The Gauss-Newton matvec is
// captured once as a CUDA graph and replayed by every PCG iteration.
//
// The Newton-Krylov method of §3.4.1 runs in lockstep: each problem keeps its
// own iteration (gradient test, forcing term, PCG stop, Armijo step) and a
// device mask tells the kernels which problems take part in a phase; masked
// tiles and reductions return at once. Each problem's arithmetic and order of
// operations are those of reg_solve on a one-problem context with the same
// options and the spectral preconditioner P_REG, so its results are bitwise
// the same.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <limits>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "reg.h"

using namespace regnk;

namespace {

// per-problem FP64 scalars: slot kind * B + p
// (J1, J2, SLOPE adjacent: the line search reads the slope <g, s> with the
// first trial's objective)
enum LsSlot { L_J1 = 0, L_J2, L_SLOPE, L_GINF, L_G2, L_RZ, L_RZNEW, L_PQ, L_RR, L_DMX, L_DMY,
              L_NSLOTS };

struct LsError {
  reg_status s;
};

// Consecutive problems with the same grid and beta: one launch per FFT pass.
struct Group {
  int p0 = 0, count = 0;
  GridDims g;
  double beta = 0;
  float2* tw1 = nullptr;
  float2* tw2 = nullptr;
  float2* spec = nullptr;   // workspace: slots spectra
  long long slots = 0;
};

// a device segmented-reduction partition (SegView) with its arrays
struct Seg {
  SegView v{};
  int total = 0;
};

}  // namespace

struct reg_lockstep {
  int device = 0;
  cudaStream_t st = nullptr;
  cudaStream_t cap = nullptr;
  reg_options opt;
  int B = 0, nt = 0;
  float ht = 0.f;
  std::vector<int> user;          // batch position -> user index
  std::vector<int> pos;           // user index -> batch position
  std::vector<BDesc> hdesc;
  std::vector<double> beta, hh;   // per batch position
  long long NT = 0;               // points of all problems
  BDesc* ddesc = nullptr;
  int4* dtiles = nullptr;
  int ntiles = 0;
  int* dpmap = nullptr;
  int* dmask = nullptr;
  int* dw = nullptr;
  std::vector<int> hw;
  Seg seg1, seg2;                 // reductions over 1 and 2 fields per problem
  double* partial = nullptr;
  float* partialf = nullptr;
  double* dsc = nullptr;          // L_NSLOTS * B
  double* hsc = nullptr;          // pinned mirror
  float* dalpha = nullptr;        // per-problem coefficients of masked linear combinations
  float* dcoef = nullptr;         // per-problem PCG step / direction weights
  int* don = nullptr;
  std::vector<Group> groups;
  std::vector<void*> allocs;
  std::vector<std::pair<int, float2*>> tw;
  // fields (F per problem): mR, mT, delta, delta_bar, fA, fB: 1; v, cv, dX,
  // dY, vtD, b, Av and the Krylov vectors: 2; m: nt + 1; gm: 2 (nt + 1); G: 2 nt
  float *mR = nullptr, *mT = nullptr, *delta = nullptr, *delta_bar = nullptr, *fA = nullptr,
        *fB = nullptr;
  float *v = nullptr, *cv = nullptr, *dX = nullptr, *dY = nullptr, *vtD = nullptr, *b = nullptr,
        *Av = nullptr;
  float *m = nullptr, *gm = nullptr, *G = nullptr;
  float *vcur = nullptr, *vtrial = nullptr, *gcur = nullptr, *kx = nullptr, *kr = nullptr,
        *kz = nullptr, *kp = nullptr, *kq = nullptr, *rhs = nullptr, *wv = nullptr, *wo = nullptr;
  bool have_images = false;
  bool have_gm = false, have_G = false;
  // the matvec graph (kp -> kq, or wv -> wo for reg_lockstep_hessian_matvec)
  struct GraphEntry {
    const float* in;
    float* out;
    int calls;
    cudaGraphExec_t exec;
    long long kernels;
  };
  std::vector<GraphEntry> graphs;
  std::vector<int> mask_now;
  std::vector<cudaStream_t> side;   // streams of the FFT runs
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  std::string err;
};

namespace {

void fail(reg_lockstep* L, reg_status s, const std::string& msg) {
  L->err = msg;
  throw LsError{s};
}

void check(reg_lockstep* L, cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(L, e == cudaErrorMemoryAllocation ? REG_ENOMEM : REG_ECUDA,
                             std::string(what) + ": " + cudaGetErrorString(e));
}

void check_launch(reg_lockstep* L, const char* what) { check(L, cudaGetLastError(), what); }

template <typename T>
T* dalloc(reg_lockstep* L, size_t n) {
  void* p = nullptr;
  check(L, cudaMalloc(&p, n * sizeof(T) + 16), "cudaMalloc");
  L->allocs.push_back(p);
  return static_cast<T*>(p);
}

float2* twiddles(reg_lockstep* L, int n) {
  for (auto& e : L->tw)
    if (e.first == n) return e.second;
  std::vector<float2> h(n);
  for (int k = 0; k < n; ++k) {
    const double a = -2.0 * M_PI * (double)k / (double)n;
    h[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  float2* d = dalloc<float2>(L, n);
  check(L, cudaMemcpy(d, h.data(), n * sizeof(float2), cudaMemcpyHostToDevice), "twiddles");
  L->tw.push_back({n, d});
  return d;
}

BRef R(float* base, int F, int k = 0) { return BRef{base, F, k}; }

BatchView view(const reg_lockstep* L) {
  BatchView v;
  v.desc = L->ddesc;
  v.w = L->dw;
  v.mask = L->dmask;
  v.tiles = L->dtiles;
  v.pmap = L->dpmap;
  v.ntiles = L->ntiles;
  return v;
}

double* slot(reg_lockstep* L, int kind) { return L->dsc + (size_t)kind * L->B; }
double hslot(const reg_lockstep* L, int kind, int p) { return L->hsc[(size_t)kind * L->B + p]; }

// Sets the device mask (problems taking part in the next phase). The source
// is pageable host memory, which cudaMemcpyAsync copies out before it
// returns, so the vector may change right after.
void set_mask(reg_lockstep* L, const std::vector<int>& mk) {
  if (mk == L->mask_now) return;
  L->mask_now = mk;
  check(L, cudaMemcpyAsync(L->dmask, mk.data(), mk.size() * sizeof(int), cudaMemcpyHostToDevice,
                           L->st), "mask");
}

void read_slots(reg_lockstep* L, int first, int count, bool with_w = false) {
  check(L, cudaMemcpyAsync(L->hsc + (size_t)first * L->B, L->dsc + (size_t)first * L->B,
                           (size_t)count * L->B * sizeof(double), cudaMemcpyDeviceToHost, L->st),
        "scalar read");
  if (with_w)
    check(L, cudaMemcpyAsync(L->hw.data(), L->dw, L->B * sizeof(int), cudaMemcpyDeviceToHost, L->st),
          "box width read");
  check(L, cudaStreamSynchronize(L->st), "synchronize");
}

// The runs of equal grids transform concurrently: run g's passes go to side
// stream g % kSideStreams, forked from and joined back to the batch's stream
// with events (graph branches under capture).
constexpr int kSideStreams = 8;

void fork_groups(reg_lockstep* L) {
  check(L, cudaEventRecord(L->ev_fork, L->st), "fork");
  for (size_t k = 0; k < L->side.size(); ++k)
    check(L, cudaStreamWaitEvent(L->side[k], L->ev_fork, 0), "fork");
}

void join_groups(reg_lockstep* L) {
  for (size_t k = 0; k < L->side.size(); ++k) {
    check(L, cudaEventRecord(L->ev_join[k], L->side[k]), "join");
    check(L, cudaStreamWaitEvent(L->st, L->ev_join[k], 0), "join");
  }
}

cudaStream_t group_stream(const reg_lockstep* L, size_t g) { return L->side[g % L->side.size()]; }

// The forward half of out = op(in) [+ add] (row R2C and column passes) for
// every problem: the arrays hold Fin fields per problem, each problem Fin /
// fin groups of fin fields; the spectra stay in the runs' workspaces for
// spectral_inv. Fields of problems outside the mask are skipped (their
// outputs are not read before the problem's next phase recomputes them).
void spectral_fwd(reg_lockstep* L, int op, double s, const float* in, int Fin, int fin, int fout) {
  fork_groups(L);
  for (size_t gi = 0; gi < L->groups.size(); ++gi) {
    const Group& g = L->groups[gi];
    const cudaStream_t st = group_stream(L, gi);
    const long long off = L->hdesc[g.p0].off;
    const int ng = g.count * (Fin / fin);
    float2* sin = g.spec;
    float2* sout = g.spec + (size_t)ng * fin * g.g.spec;
    const FieldMask fmi{L->dmask, g.p0, Fin}, fmc{L->dmask, g.p0, Fin / fin};
    fft_rows_r2c(g.g.n1, g.g.n2, in + (size_t)Fin * off, g.g.N, sin, g.g.spec, ng * fin, g.tw1, st,
                 fmi);
    ColArgs a{};
    a.n1_in = a.n1_out = a.n1 = g.g.n1;
    a.n2_in = a.n2_out = a.n2 = g.g.n2;
    a.nk1_out = g.g.nk1;
    a.op = op;
    a.beta = (float)g.beta;
    a.p = L->opt.reg_norm;
    a.s = (float)s;
    a.beta_w = 0.f;
    a.scale = (float)(1.0 / (double)g.g.N);
    a.tw_in = a.tw_out = g.tw2;
    a.in = sin;
    a.in_fstride = g.g.spec;
    a.out = sout;
    a.out_fstride = g.g.spec;
    a.nin = fin;
    a.nout = fout;
    a.fm = fmc;
    fft_cols(a, ng, st);
  }
  check_launch(L, "spectral operator");
}

// The inverse half: row C2R passes of the spectra spectral_fwd left, with the
// addend, after everything queued on the batch's stream; joins the runs'
// streams back.
void spectral_inv(reg_lockstep* L, int Fin, int fin, float* out, int Fout, int fout,
                  const float* add) {
  fork_groups(L);
  for (size_t gi = 0; gi < L->groups.size(); ++gi) {
    const Group& g = L->groups[gi];
    const cudaStream_t st = group_stream(L, gi);
    const long long off = L->hdesc[g.p0].off;
    const int ng = g.count * (Fin / fin);
    float2* sout = g.spec + (size_t)ng * fin * g.g.spec;
    const FieldMask fmo{L->dmask, g.p0, Fout};
    fft_rows_c2r(g.g.n1, g.g.n2, sout, g.g.spec, out + (size_t)Fout * off, g.g.N,
                 add ? add + (size_t)Fout * off : nullptr, g.g.N, ng * fout, g.tw1, st, nullptr,
                 fmo);
  }
  join_groups(L);
  check_launch(L, "spectral operator");
}

// out (Fout fields per problem) = op(in (Fin fields per problem)) [+ add]
void spectral(reg_lockstep* L, int op, double s, const float* in, int Fin, int fin, float* out,
              int Fout, int fout, const float* add) {
  spectral_fwd(L, op, s, in, Fin, fin, fout);
  spectral_inv(L, Fin, fin, out, Fout, fout, add);
}

void dot(reg_lockstep* L, BRef a, BRef b, int len, int kind) {
  const Seg& S = len == 1 ? L->seg1 : L->seg2;
  launch_dot_b(L->ddesc, S.v, L->B, L->dmask, a, b, len, L->partial, slot(L, kind), L->st);
}

// Caches v (2 fields per problem), its characteristics, the box widths of
// the fused kernels and the state history m_0..m_nt (§3.3.2) for the
// problems of the mask.
void set_velocity(reg_lockstep* L, const float* v) {
  const BatchView V = view(L);
  const int nt = L->nt;
  const int Fm = nt + 1;
  if (v != L->v)
    check(L, cudaMemcpyAsync(L->v, v, 2 * L->NT * sizeof(float), cudaMemcpyDeviceToDevice, L->st),
          "copy v");
  launch_prefilter_b(V, R(L->v, 2), R(L->cv, 2), 2, L->st);
  launch_departure_b(V, L->NT, R(L->v, 2), R(L->cv, 2), R(L->dX, 2), R(L->dY, 2), L->st);
  launch_maxabs_b(L->ddesc, L->seg2.v, L->B, L->dmask, R(L->dX, 2), 2, L->partialf,
                  slot(L, L_DMX), L->st);
  launch_maxabs_b(L->ddesc, L->seg2.v, L->B, L->dmask, R(L->dY, 2), 2, L->partialf,
                  slot(L, L_DMY), L->st);
  launch_set_w_b(L->B, slot(L, L_DMX), slot(L, L_DMY), L->dw, L->st);
  launch_copy_field_b(V, L->NT, R(L->mT, 1), R(L->m, Fm, 0), L->st);
  for (int j = 1; j <= nt; ++j)
    launch_gather_fused_b(V, R(L->m, Fm, j - 1), 1, R(L->dX, 2), R(L->m, Fm, j), L->st);
  check_launch(L, "state solve");
  spectral(L, SPOP_DIV, 0.0, L->v, 2, 2, L->delta, 1, 1, nullptr);
  launch_gather_fused_b(V, R(L->delta, 1), 1, R(L->dY, 2), R(L->delta_bar, 1), L->st);
  check_launch(L, "div v");
  L->have_gm = false;
  L->have_G = false;
}

void ensure_grad_history(reg_lockstep* L) {
  if (L->have_gm) return;
  // grad m_0..grad m_nt (grad m_0 = grad m_T again, bitwise the same)
  spectral(L, SPOP_GRAD, 0.0, L->m, L->nt + 1, 1, L->gm, 2 * (L->nt + 1), 2, nullptr);
  L->have_gm = true;
}

void ensure_G(reg_lockstep* L) {
  if (L->have_G) return;
  ensure_grad_history(L);
  const BatchView V = view(L);
  const int Fg = 2 * (L->nt + 1), FG = 2 * L->nt;
  for (int j = 1; j <= L->nt; ++j)
    launch_gather_fused_b(V, R(L->gm, Fg, 2 * (j - 1)), 2, R(L->dX, 2), R(L->G, FG, 2 * (j - 1)),
                          L->st);
  check_launch(L, "G history");
  L->have_G = true;
}

// J_p = 1/2 <m_1 - m_R, m_1 - m_R>_h + beta/2 <v, A v>_h (eq. varopt:objective)
// for the problems of the mask (+inf where a displacement exceeds the fused
// kernels' box); leaves beta A v in Av.
std::vector<double> objective(reg_lockstep* L) {
  spectral(L, SPOP_REGPOW, 1.0, L->v, 2, 1, L->Av, 2, 1, nullptr);
  const Seg& S1 = L->seg1;
  launch_sumsq_diff_b(L->ddesc, S1.v, L->B, L->dmask, R(L->m, L->nt + 1, L->nt), R(L->mR, 1), 1,
                      L->partial, slot(L, L_J1), L->st);
  dot(L, R(L->v, 2), R(L->Av, 2), 2, L_J2);
  check_launch(L, "objective");
  read_slots(L, L_J1, 3, true);
  std::vector<double> J(L->B);
  for (int p = 0; p < L->B; ++p) {
    const double hh = L->hh[p];
    J[p] = L->hw[p] ? 0.5 * hh * hslot(L, L_J1, p) + 0.5 * hh * hslot(L, L_J2, p)
                    : std::numeric_limits<double>::infinity();
  }
  return J;
}

// g = beta A v + b, b = int_0^1 lambda grad m dt by the adjoint solve
// (eq. adj-slm); needs objective() for Av.
void gradient(reg_lockstep* L, float* g_out) {
  ensure_grad_history(L);
  const BatchView V = view(L);
  const int nt = L->nt;
  const float ht = L->ht;
  const int Fg = 2 * (nt + 1);
  float* lam = L->fA;
  float* lam2 = L->fB;
  launch_adjoint_init_b(V, L->NT, 0.5f * ht, R(L->mR, 1), R(L->m, nt + 1, nt), R(L->gm, Fg, 2 * nt),
                        R(lam, 1), R(L->b, 2), 1.f, L->st);
  for (int j = nt - 1; j >= 0; --j) {
    const float wb = ht * (j == 0 ? 0.5f : 1.0f);
    launch_adjoint_fused_b(V, ht, wb, R(lam, 1), R(L->dY, 2), R(L->delta, 1), R(L->delta_bar, 1),
                           R(L->gm, Fg, 2 * j), R(lam2, 1), R(L->b, 2), L->st);
    std::swap(lam, lam2);
  }
  check_launch(L, "adjoint solve");
  launch_lincomb(2 * L->NT, 1.f, L->Av, 1.f, L->b, g_out, L->st);
  check_launch(L, "gradient");
}

// Gauss-Newton Hessian matvec (eq. hessian-matvec, GN) of every problem:
// the incremental state forward, the incremental adjoint backward with
// b~ = int lambda~ grad m dt, then beta A v~ + b~ (eq. inc-state-slm,
// eq. inc-adj-slm).
void hessian(reg_lockstep* L, const float* vt, float* out) {
  const BatchView V = view(L);
  const int nt = L->nt;
  const float ht = L->ht;
  const int Fg = 2 * (nt + 1), FG = 2 * nt;
  float* mt = L->fA;
  float* mt2 = L->fB;
  float* vtm = const_cast<float*>(vt);
  // beta A v~: its forward transforms depend only on v~ and run on the runs'
  // streams while the transport steps (which use no FFT workspace) run here
  spectral_fwd(L, SPOP_REGPOW, 1.0, vt, 2, 1, 1);
  launch_incstate_first_fused_b(V, ht, R(vtm, 2), R(L->dX, 2), R(L->G, FG, 0), R(L->gm, Fg, 2),
                                R(L->vtD, 2), R(mt2, 1), L->st);
  std::swap(mt, mt2);
  for (int j = 2; j <= nt; ++j) {
    const bool last = (j == nt);
    launch_incstate_fused_b(V, ht, R(mt, 1), R(L->dX, 2), R(vtm, 2), R(L->vtD, 2),
                            R(L->G, FG, 2 * (j - 1)), R(L->gm, Fg, 2 * j), R(mt2, 1),
                            last ? R(L->gm, Fg, 2 * nt) : R(nullptr, 1),
                            last ? R(L->b, 2) : R(nullptr, 2), L->st);
    std::swap(mt, mt2);
  }
  check_launch(L, "incremental state");
  float* lt = mt;
  float* lt2 = mt2;
  if (nt < 2) {   // lambda~_nt = -m~_nt and the first term of b~
    lt = mt2;
    launch_adjoint_init_b(V, L->NT, 0.5f * ht, R(nullptr, 1), R(mt, 1), R(L->gm, Fg, 2 * nt),
                          R(lt, 1), R(L->b, 2), 1.f, L->st);
    lt2 = mt;
  }
  for (int j = nt - 1; j >= 0; --j) {
    const float wb = ht * (j == 0 ? 0.5f : 1.0f);
    launch_adjoint_fused_b(V, ht, wb, R(lt, 1), R(L->dY, 2), R(L->delta, 1), R(L->delta_bar, 1),
                           R(L->gm, Fg, 2 * j), R(lt2, 1), R(L->b, 2), L->st);
    std::swap(lt, lt2);
  }
  check_launch(L, "incremental adjoint");
  spectral_inv(L, 2, 1, out, 2, 1, L->b);
}

// The matvec in -> out of every problem of the mask, captured as a CUDA
// graph on its second call with these buffers and replayed from the third
// (the mask and the box widths are device data the graph reads).
void matvec(reg_lockstep* L, const float* in, float* out) {
  reg_lockstep::GraphEntry* e = nullptr;
  for (auto& g : L->graphs)
    if (g.in == in && g.out == out) e = &g;
  if (!e) {
    L->graphs.push_back({in, out, 0, nullptr, 0});
    e = &L->graphs.back();
  }
  if (!L->opt.use_graphs || e->calls < 1) {
    ++e->calls;
    hessian(L, in, out);
    return;
  }
  if (!e->exec) {
    cudaStream_t user = L->st;
    const int saved = t_programmatic_launch;
    check(L, cudaStreamBeginCapture(L->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    L->st = L->cap;
    t_programmatic_launch = 0;   // plain launches inside the graph
    cudaGraph_t graph = nullptr;
    try {
      hessian(L, in, out);
    } catch (...) {
      cudaStreamEndCapture(L->cap, &graph);
      if (graph) cudaGraphDestroy(graph);
      L->st = user;
      t_programmatic_launch = saved;
      cudaGetLastError();
      throw;
    }
    L->st = user;
    t_programmatic_launch = saved;
    check(L, cudaStreamEndCapture(L->cap, &graph), "end capture");
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
    long long kn = 0;
    for (size_t i = 0; i < nn; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
    }
    e->kernels = kn;
    g_launch_count -= kn;
    const cudaError_t ie = cudaGraphInstantiate(&e->exec, graph, 0);
    cudaGraphDestroy(graph);
    check(L, ie, "graph instantiate");
  }
  ++e->calls;
  check(L, cudaGraphLaunch(e->exec, L->st), "graph launch");
  g_launch_count += e->kernels;
}

// P_REG (§3.4.2): z = (beta A)^-1 r
void precond(reg_lockstep* L, const float* r, float* z) {
  spectral(L, SPOP_REGPOW, -1.0, r, 2, 1, z, 2, 1, nullptr);
}

std::vector<int> all_of(int B, int v = 1) { return std::vector<int>(B, v); }

// per-problem result of a lockstep PCG
struct PcgOut {
  std::vector<int> iters, matvecs;
};

// PCG (Hestenes-Stiefel) from x = 0 on the problems of `act`, each with its
// own tolerance: the same steps as the one-problem PCG, every vector
// operation masked to the problems still iterating. bb[p] = <rhs, rhs> of
// problem p (the right-hand side -g has the squared norm <g, g> the Newton
// loop already holds, to the bit).
PcgOut pcg(reg_lockstep* L, const std::vector<int>& act, const std::vector<double>& rtol,
           const std::vector<double>& bb, int maxit) {
  const int B = L->B;
  const long long n = 2 * L->NT;
  PcgOut out;
  out.iters.assign(B, 0);
  out.matvecs.assign(B, 0);
  std::vector<int> run = act;
  set_mask(L, run);
  launch_fill(L->kx, n, 0.f, L->st);
  check(L, cudaMemcpyAsync(L->kr, L->rhs, n * sizeof(float), cudaMemcpyDeviceToDevice, L->st), "copy");
  std::vector<double> bnorm(B, 0.0);
  for (int p = 0; p < B; ++p) {
    if (!run[p]) continue;
    bnorm[p] = std::sqrt(bb[p]);
    if (!(bnorm[p] > 0.0)) run[p] = 0;
  }
  if (std::none_of(run.begin(), run.end(), [](int x) { return x != 0; })) return out;
  set_mask(L, run);
  precond(L, L->kr, L->kz);
  check(L, cudaMemcpyAsync(L->kp, L->kz, n * sizeof(float), cudaMemcpyDeviceToDevice, L->st), "copy");
  dot(L, R(L->kr, 2), R(L->kz, 2), 2, L_RZ);
  for (int it = 0; it < maxit; ++it) {
    matvec(L, L->kp, L->kq);
    for (int p = 0; p < B; ++p)
      if (run[p]) ++out.matvecs[p];
    dot(L, R(L->kp, 2), R(L->kq, 2), 2, L_PQ);
    launch_pcg_update_b(L->dpmap, L->dmask, B, 2, n, slot(L, L_RZ), slot(L, L_PQ), L->dcoef, L->don,
                        L->kp, L->kq, L->kx, L->kr, L->st);
    dot(L, R(L->kr, 2), R(L->kr, 2), 2, L_RR);
    read_slots(L, L_PQ, 2);
    std::vector<int> next = run;
    for (int p = 0; p < B; ++p) {
      if (!run[p]) continue;
      const double pq = hslot(L, L_PQ, p), rr = hslot(L, L_RR, p);
      if (!(pq > 0.0)) {   // negative curvature: x and r were left unchanged
        if (it == 0) {
          const size_t o = 2 * (size_t)L->hdesc[p].off, len = 2 * (size_t)L->hdesc[p].n1 * L->hdesc[p].n2;
          check(L, cudaMemcpyAsync(L->kx + o, L->kz + o, len * sizeof(float),
                                   cudaMemcpyDeviceToDevice, L->st), "copy");
        }
        next[p] = 0;
        continue;
      }
      out.iters[p] = it + 1;
      if (std::sqrt(rr) / bnorm[p] <= rtol[p]) next[p] = 0;
    }
    run = next;
    if (std::none_of(run.begin(), run.end(), [](int x) { return x != 0; })) break;
    set_mask(L, run);
    precond(L, L->kr, L->kz);
    dot(L, R(L->kr, 2), R(L->kz, 2), 2, L_RZNEW);
    launch_pcg_direction_b(L->dpmap, L->dmask, B, 2, n, slot(L, L_RZNEW), slot(L, L_RZ), L->dcoef,
                           L->don, L->kz, L->kp, L->st);
    launch_copy_scalars_b(B, L->dmask, slot(L, L_RZNEW), slot(L, L_RZ), L->st);
    check_launch(L, "pcg");
  }
  return out;
}

// masked z = a_p x + b_p y with per-problem coefficients given on the host
void lincomb_masked(reg_lockstep* L, const std::vector<float>& a, const float* x,
                    const std::vector<float>& bc, const float* y, float* z) {
  std::vector<float> h(2 * L->B);
  std::copy(a.begin(), a.end(), h.begin());
  std::copy(bc.begin(), bc.end(), h.begin() + L->B);
  check(L, cudaMemcpyAsync(L->dalpha, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice,
                           L->st), "coefficients");
  launch_lincomb_b(L->dpmap, L->dmask, 2, 2 * L->NT, L->dalpha, x, L->dalpha + L->B, y, z, L->st);
  check_launch(L, "lincomb");
}

void copy_in(reg_lockstep* L, float* dst, const float* const* src, int F) {
  for (int p = 0; p < L->B; ++p) {
    const BDesc& D = L->hdesc[p];
    const size_t len = (size_t)F * D.n1 * D.n2;
    check(L, cudaMemcpyAsync(dst + (size_t)F * D.off, src[L->user[p]], len * sizeof(float),
                             cudaMemcpyDeviceToDevice, L->st), "copy in");
  }
}

void copy_out(reg_lockstep* L, float* const* dst, const float* src, int F) {
  for (int p = 0; p < L->B; ++p) {
    const BDesc& D = L->hdesc[p];
    const size_t len = (size_t)F * D.n1 * D.n2;
    check(L, cudaMemcpyAsync(dst[L->user[p]], src + (size_t)F * D.off, len * sizeof(float),
                             cudaMemcpyDeviceToDevice, L->st), "copy out");
  }
}

reg_status guarded(reg_lockstep* L, const std::function<void()>& body) {
  if (!L) return REG_EINVAL;
  const int saved_mode = t_programmatic_launch;
  const int saved_prec = t_plain_fp32_reduce;
  t_programmatic_launch = L->opt.programmatic_launch ? 1 : 0;
  t_plain_fp32_reduce = 0;
  reg_status s = REG_OK;
  try {
    body();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      L->err = std::string("CUDA: ") + cudaGetErrorString(e);
      s = REG_ECUDA;
    }
  } catch (const LsError& e) {
    s = e.s;
  }
  t_programmatic_launch = saved_mode;
  t_plain_fp32_reduce = saved_prec;
  return s;
}

bool size_ok(int n) { return n % 32 == 0 && fft_size_supported(n); }

bool unaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

}  // namespace

extern "C" {

reg_status reg_lockstep_create(const reg_grid* grids, int B, int nt, const double* beta,
                               const reg_options* opt, reg_lockstep** out) {
  if (!out || !grids || !beta || B < 1 || B > 4096 || nt < 1 || nt > 4096) return REG_EINVAL;
  *out = nullptr;
  reg_options o;
  if (opt) o = *opt; else reg_default_options(&o);
  // the lockstep form runs the fused spline path with the spectral
  // preconditioner, the Gauss-Newton matvec and FP64-accurate reductions
  if (o.reg_norm < 1 || o.reg_norm > 3 || o.interp != REG_INTERP_SPLINE || o.precond != REG_PC_REG ||
      o.hessian != REG_HESSIAN_GN || o.precision != REG_PRECISION_FP64 || o.incompressible ||
      o.beta_w != 0.0 || !o.fused_transport || o.persistent_matvec || o.max_pcg < 1 ||
      o.max_newton < 0 || (o.use_graphs != 0 && o.use_graphs != 1))
    return REG_EINVAL;
  for (int i = 0; i < B; ++i)
    if (!size_ok(grids[i].n1) || !size_ok(grids[i].n2) || !(beta[i] > 0.0)) return REG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return REG_ECUDA;
  reg_lockstep* L = new reg_lockstep();
  L->device = dev;
  L->opt = o;
  L->B = B;
  L->nt = nt;
  L->ht = 1.0f / (float)nt;
  // batch order: largest grids first (their tiles start first), problems with
  // the same grid and beta adjacent (one FFT launch per pass for each run)
  L->user.resize(B);
  std::iota(L->user.begin(), L->user.end(), 0);
  std::stable_sort(L->user.begin(), L->user.end(), [&](int a, int b) {
    const long long na = (long long)grids[a].n1 * grids[a].n2, nb = (long long)grids[b].n1 * grids[b].n2;
    if (na != nb) return na > nb;
    if (grids[a].n1 != grids[b].n1) return grids[a].n1 > grids[b].n1;
    return beta[a] < beta[b];
  });
  L->pos.resize(B);
  for (int p = 0; p < B; ++p) L->pos[L->user[p]] = p;
  const reg_status s = guarded(L, [&] {
    check(L, cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking), "stream");
    check(L, cudaStreamCreateWithFlags(&L->cap, cudaStreamNonBlocking), "capture stream");
    batch_fused_init();
    long long off = 0;
    std::vector<int4> tiles;
    std::vector<int> pmap;
    for (int p = 0; p < B; ++p) {
      const reg_grid gr = grids[L->user[p]];
      const GridDims g = make_grid(gr.n1, gr.n2);
      BDesc D;
      D.n1 = gr.n1;
      D.n2 = gr.n2;
      D.p2 = (g.log1 >= 0 && g.log2 >= 0);
      D.log1 = D.p2 ? g.log1 : -1;
      D.off = off;
      D.s1 = departure_scale(L->ht, gr.n1);
      D.s2 = departure_scale(L->ht, gr.n2);
      L->hdesc.push_back(D);
      L->beta.push_back(beta[L->user[p]]);
      L->hh.push_back((2.0 * M_PI / gr.n1) * (2.0 * M_PI / gr.n2));
      for (int ty = 0; ty < gr.n2 / 32; ++ty)
        for (int tx = 0; tx < gr.n1 / 32; ++tx) tiles.push_back(make_int4(p, tx, ty, 0));
      for (long long k = 0; k < g.N / 1024; ++k) pmap.push_back(p);
      off += g.N;
    }
    L->NT = off;
    L->ntiles = (int)tiles.size();
    L->ddesc = dalloc<BDesc>(L, B);
    check(L, cudaMemcpy(L->ddesc, L->hdesc.data(), B * sizeof(BDesc), cudaMemcpyHostToDevice), "desc");
    L->dtiles = dalloc<int4>(L, tiles.size());
    check(L, cudaMemcpy(L->dtiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice),
          "tiles");
    L->dpmap = dalloc<int>(L, pmap.size());
    check(L, cudaMemcpy(L->dpmap, pmap.data(), pmap.size() * sizeof(int), cudaMemcpyHostToDevice), "pmap");
    // segmented reductions over 1 and 2 fields per problem
    int maxblocks = 0;
    for (int len = 1; len <= 2; ++len) {
      std::vector<int2> blocks;
      std::vector<int> nb(B), first(B);
      for (int p = 0; p < B; ++p) {
        const long long n = (long long)len * L->hdesc[p].n1 * L->hdesc[p].n2;
        nb[p] = reduce_blocks(n);
        first[p] = (int)blocks.size();
        for (int k = 0; k < nb[p]; ++k) blocks.push_back(make_int2(p, k));
      }
      Seg& S = len == 1 ? L->seg1 : L->seg2;
      int2* db = dalloc<int2>(L, blocks.size());
      int* dnb = dalloc<int>(L, B);
      int* dfirst = dalloc<int>(L, B);
      check(L, cudaMemcpy(db, blocks.data(), blocks.size() * sizeof(int2), cudaMemcpyHostToDevice), "seg");
      check(L, cudaMemcpy(dnb, nb.data(), B * sizeof(int), cudaMemcpyHostToDevice), "seg");
      check(L, cudaMemcpy(dfirst, first.data(), B * sizeof(int), cudaMemcpyHostToDevice), "seg");
      S.v.blocks = db;
      S.v.nb = dnb;
      S.v.first = dfirst;
      S.v.nblocks = (int)blocks.size();
      S.total = (int)blocks.size();
      maxblocks = std::max(maxblocks, S.total);
    }
    L->partial = dalloc<double>(L, maxblocks);
    L->partialf = dalloc<float>(L, maxblocks);
    L->dmask = dalloc<int>(L, B);
    L->mask_now = all_of(B);
    check(L, cudaMemcpy(L->dmask, L->mask_now.data(), B * sizeof(int), cudaMemcpyHostToDevice), "mask");
    L->dw = dalloc<int>(L, B);
    check(L, cudaMemset(L->dw, 0, B * sizeof(int)), "memset");
    L->hw.assign(B, 0);
    L->dsc = dalloc<double>(L, (size_t)L_NSLOTS * B);
    void* h = nullptr;
    check(L, cudaMallocHost(&h, (size_t)L_NSLOTS * B * sizeof(double)), "cudaMallocHost");
    L->hsc = static_cast<double*>(h);
    L->dalpha = dalloc<float>(L, 2 * B);
    L->dcoef = dalloc<float>(L, B);
    L->don = dalloc<int>(L, B);
    // FFT groups
    for (int p = 0; p < B;) {
      Group g;
      g.p0 = p;
      const BDesc& D = L->hdesc[p];
      int q = p;
      while (q < B && L->hdesc[q].n1 == D.n1 && L->hdesc[q].n2 == D.n2 && L->beta[q] == L->beta[p]) ++q;
      g.count = q - p;
      g.g = make_grid(D.n1, D.n2);
      g.beta = L->beta[p];
      g.tw1 = twiddles(L, D.n1);
      g.tw2 = twiddles(L, D.n2);
      g.slots = (long long)g.count * std::max(3 * (nt + 1), 4);
      g.spec = dalloc<float2>(L, (size_t)g.slots * g.g.spec);
      L->groups.push_back(g);
      p = q;
    }
    const size_t ns = std::min(L->groups.size(), (size_t)kSideStreams);
    L->side.assign(ns, nullptr);
    L->ev_join.assign(ns, nullptr);
    check(L, cudaEventCreateWithFlags(&L->ev_fork, cudaEventDisableTiming), "event");
    for (size_t k = 0; k < ns; ++k) {
      check(L, cudaStreamCreateWithFlags(&L->side[k], cudaStreamNonBlocking), "stream");
      check(L, cudaEventCreateWithFlags(&L->ev_join[k], cudaEventDisableTiming), "event");
    }
    const size_t N = (size_t)L->NT;
    L->mR = dalloc<float>(L, N);
    L->mT = dalloc<float>(L, N);
    L->delta = dalloc<float>(L, N);
    L->delta_bar = dalloc<float>(L, N);
    L->fA = dalloc<float>(L, N);
    L->fB = dalloc<float>(L, N);
    float** vec[] = {&L->v, &L->cv, &L->dX, &L->dY, &L->vtD, &L->b, &L->Av, &L->vcur, &L->vtrial,
                     &L->gcur, &L->kx, &L->kr, &L->kz, &L->kp, &L->kq, &L->rhs, &L->wv, &L->wo};
    for (float** f : vec) *f = dalloc<float>(L, 2 * N);
    L->m = dalloc<float>(L, (size_t)(nt + 1) * N);
    L->gm = dalloc<float>(L, 2 * (size_t)(nt + 1) * N);
    L->G = dalloc<float>(L, 2 * (size_t)nt * N);
    check(L, cudaDeviceSynchronize(), "create");
  });
  if (s != REG_OK) {
    reg_lockstep_destroy(L);
    return s;
  }
  *out = L;
  return REG_OK;
}

reg_status reg_lockstep_destroy(reg_lockstep* L) {
  if (!L) return REG_OK;
  if (L->st) cudaStreamSynchronize(L->st);
  for (auto& g : L->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (void* p : L->allocs) cudaFree(p);
  if (L->hsc) cudaFreeHost(L->hsc);
  for (cudaStream_t x : L->side)
    if (x) cudaStreamDestroy(x);
  for (cudaEvent_t e : L->ev_join)
    if (e) cudaEventDestroy(e);
  if (L->ev_fork) cudaEventDestroy(L->ev_fork);
  if (L->cap) cudaStreamDestroy(L->cap);
  if (L->st) cudaStreamDestroy(L->st);
  delete L;
  return REG_OK;
}

reg_status reg_lockstep_set_stream(reg_lockstep* L, void* stream) {
  if (!L) return REG_EINVAL;
  // the batch keeps its own stream; the caller's stream is ordered before it
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return REG_ECUDA;
  cudaEventRecord(ev, user);
  cudaStreamWaitEvent(L->st, ev, 0);
  cudaEventDestroy(ev);
  return cudaGetLastError() == cudaSuccess ? REG_OK : REG_ECUDA;
}

reg_status reg_lockstep_set_images(reg_lockstep* L, const float* const* m_R,
                                   const float* const* m_T) {
  if (!L || !m_R || !m_T) return REG_EINVAL;
  for (int i = 0; i < L->B; ++i)
    if (!m_R[i] || !m_T[i] || unaligned(m_R[i]) || unaligned(m_T[i])) return REG_EINVAL;
  return guarded(L, [&] {
    copy_in(L, L->mR, m_R, 1);
    copy_in(L, L->mT, m_T, 1);
    L->have_images = true;
    L->have_gm = L->have_G = false;
    check(L, cudaStreamSynchronize(L->st), "synchronize");
  });
}

reg_status reg_lockstep_objective_gradient(reg_lockstep* L, const float* const* v, double* J,
                                           float* const* g) {
  if (!L || !v || !J) return REG_EINVAL;
  return guarded(L, [&] {
    if (!L->have_images) fail(L, REG_ESTATE, "reg_lockstep_set_images has not been called");
    set_mask(L, all_of(L->B));
    copy_in(L, L->vcur, v, 2);
    set_velocity(L, L->vcur);
    const std::vector<double> Jb = objective(L);
    for (int p = 0; p < L->B; ++p) J[L->user[p]] = Jb[p];
    if (g) {
      gradient(L, L->gcur);
      copy_out(L, g, L->gcur, 2);
    }
    check(L, cudaStreamSynchronize(L->st), "synchronize");
    for (int p = 0; p < L->B; ++p)
      if (!L->hw[p])
        fail(L, REG_EINVAL, "problem " + std::to_string(L->user[p]) +
                                ": displacement per step beyond the fused kernels' 14 cells");
  });
}

reg_status reg_lockstep_hessian_matvec(reg_lockstep* L, const float* const* v,
                                       const float* const* vt, float* const* Hvt) {
  if (!L || !v || !vt || !Hvt) return REG_EINVAL;
  return guarded(L, [&] {
    if (!L->have_images) fail(L, REG_ESTATE, "reg_lockstep_set_images has not been called");
    set_mask(L, all_of(L->B));
    copy_in(L, L->vcur, v, 2);
    set_velocity(L, L->vcur);
    check(L, cudaMemcpyAsync(L->hw.data(), L->dw, L->B * sizeof(int), cudaMemcpyDeviceToHost, L->st),
          "box width read");
    check(L, cudaStreamSynchronize(L->st), "synchronize");
    for (int p = 0; p < L->B; ++p)
      if (!L->hw[p])
        fail(L, REG_EINVAL, "problem " + std::to_string(L->user[p]) +
                                ": displacement per step beyond the fused kernels' 14 cells");
    ensure_G(L);
    copy_in(L, L->wv, vt, 2);
    matvec(L, L->wv, L->wo);
    copy_out(L, Hvt, L->wo, 2);
    check(L, cudaStreamSynchronize(L->st), "synchronize");
  });
}

reg_status reg_lockstep_solve(reg_lockstep* L, float* const* v, double gtol, reg_info* infos) {
  if (!L || !v || !(gtol > 0.0)) return REG_EINVAL;
  for (int i = 0; i < L->B; ++i)
    if (!v[i] || unaligned(v[i])) return REG_EINVAL;
  const int B = L->B;
  std::vector<reg_info> inf(B);
  for (auto& x : inf) std::memset(&x, 0, sizeof x);
  std::vector<int> status(B, REG_OK);
  const auto t0 = std::chrono::steady_clock::now();
  const long long n = 2 * L->NT;
  const reg_status s = guarded(L, [&] {
    if (!L->have_images) fail(L, REG_ESTATE, "reg_lockstep_set_images has not been called");
    const reg_options& o = L->opt;
    // reference gradient at v = 0 (the relative stopping test)
    set_mask(L, all_of(B));
    launch_fill(L->vtrial, n, 0.f, L->st);
    set_velocity(L, L->vtrial);
    objective(L);
    gradient(L, L->gcur);
    launch_maxabs_b(L->ddesc, L->seg2.v, B, L->dmask, R(L->gcur, 2), 2, L->partialf,
                    slot(L, L_GINF), L->st);
    dot(L, R(L->gcur, 2), R(L->gcur, 2), 2, L_G2);
    read_slots(L, L_GINF, 2);
    std::vector<double> gref_inf(B), gref_2(B);
    for (int p = 0; p < B; ++p) {
      gref_inf[p] = hslot(L, L_GINF, p);
      gref_2[p] = std::sqrt(hslot(L, L_G2, p));
      inf[p].gref_inf = gref_inf[p];
    }
    // J and g at the initial guess
    copy_in(L, L->vcur, v, 2);
    set_velocity(L, L->vcur);
    std::vector<double> J = objective(L);
    for (int p = 0; p < B; ++p) {
      if (!L->hw[p]) {
        status[p] = REG_EINVAL;
        L->err = "a problem's initial displacement per step exceeds the fused kernels' 14 cells";
      }
      inf[p].J0 = J[p];
    }
    gradient(L, L->gcur);
    std::vector<int> active(B);
    for (int p = 0; p < B; ++p) active[p] = (status[p] == REG_OK);
    std::vector<double> rel(B, 1.0), ginf(B, 0.0);
    for (int k = 0;; ++k) {
      set_mask(L, active);
      launch_maxabs_b(L->ddesc, L->seg2.v, B, L->dmask, R(L->gcur, 2), 2, L->partialf,
                      slot(L, L_GINF), L->st);
      dot(L, R(L->gcur, 2), R(L->gcur, 2), 2, L_G2);
      read_slots(L, L_GINF, 2);
      std::vector<double> rtol(B, 0.0), gg(B, 0.0);
      for (int p = 0; p < B; ++p) {
        if (!active[p]) continue;
        ginf[p] = hslot(L, L_GINF, p);
        if (!std::isfinite(ginf[p]) || !std::isfinite(J[p])) {
          status[p] = REG_ENONFINITE;
          active[p] = 0;
          continue;
        }
        rel[p] = ginf[p] / gref_inf[p];
        if (rel[p] <= gtol || ginf[p] <= o.gabs) { active[p] = 0; continue; }
        if (k == o.max_newton) { status[p] = REG_ENOTCONV; active[p] = 0; continue; }
        gg[p] = hslot(L, L_G2, p);
        rtol[p] = std::fmin(0.5, std::sqrt(gg[p]) / gref_2[p]);
      }
      if (std::none_of(active.begin(), active.end(), [](int x) { return x != 0; })) break;
      set_mask(L, active);
      ensure_G(L);
      launch_lincomb(n, -1.f, L->gcur, 0.f, nullptr, L->rhs, L->st);   // rhs = -g
      const PcgOut pr = pcg(L, active, rtol, gg, o.max_pcg);
      for (int p = 0; p < B; ++p) {
        inf[p].pcg_iters += pr.iters[p];
        inf[p].matvecs += pr.matvecs[p];
      }
      set_mask(L, active);
      dot(L, R(L->gcur, 2), R(L->kx, 2), 2, L_SLOPE);   // read with the first trial's J
      std::vector<double> slope(B, 0.0), alpha(B, 1.0), Jt(B, 0.0);
      std::vector<int> search = active, accepted(B, 0);
      for (int ls = 0; ls <= o.max_backtracks; ++ls) {
        set_mask(L, search);
        std::vector<float> a(B, 1.f), al(B, 0.f);
        for (int p = 0; p < B; ++p) al[p] = (float)alpha[p];
        lincomb_masked(L, a, L->vcur, al, L->kx, L->vtrial);
        set_velocity(L, L->vtrial);
        const std::vector<double> Jl = objective(L);
        if (ls == 0)
          for (int p = 0; p < B; ++p) slope[p] = L->hh[p] * hslot(L, L_SLOPE, p);
        for (int p = 0; p < B; ++p) {
          if (!search[p]) continue;
          Jt[p] = Jl[p];
          ++inf[p].line_search_steps;
          if (Jt[p] <= J[p] + o.armijo_c1 * alpha[p] * slope[p]) {
            accepted[p] = 1;
            search[p] = 0;
          } else {
            alpha[p] *= 0.5;
          }
        }
        if (std::none_of(search.begin(), search.end(), [](int x) { return x != 0; })) break;
      }
      for (int p = 0; p < B; ++p)
        if (active[p] && !accepted[p]) {
          status[p] = REG_ELINESEARCH;
          active[p] = 0;
        }
      // accept: v = v_trial; J; the gradient at the accepted velocity (the
      // cached state of every accepted problem is its accepted trial)
      set_mask(L, accepted);
      {
        std::vector<float> one(B, 1.f), zero(B, 0.f);
        lincomb_masked(L, one, L->vtrial, zero, nullptr, L->vcur);
      }
      for (int p = 0; p < B; ++p)
        if (accepted[p]) {
          J[p] = Jt[p];
          ++inf[p].newton_iters;
        }
      if (std::any_of(accepted.begin(), accepted.end(), [](int x) { return x != 0; })) {
        // the cached state holds the accepted trials, but its gradient
        // history and G belong to the last trial of each problem: rebuilt
        L->have_gm = L->have_G = false;
        gradient(L, L->gcur);
      }
    }
    for (int p = 0; p < B; ++p) {
      inf[p].J = J[p];
      inf[p].gnorm_rel = rel[p];
      inf[p].gnorm_inf = ginf[p];
    }
    set_mask(L, all_of(B));
    copy_out(L, v, L->vcur, 2);
    check(L, cudaStreamSynchronize(L->st), "synchronize");
  });
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  reg_status worst = REG_OK;
  for (int p = 0; p < B; ++p) {
    inf[p].seconds = secs;
    inf[p].status = (s != REG_OK) ? s : status[p];
    if (infos) infos[L->user[p]] = inf[p];
    if (status[p] == REG_OK) continue;
    if ((status[p] == REG_ENOTCONV || status[p] == REG_ELINESEARCH) && worst == REG_OK)
      worst = (reg_status)status[p];
    else if (status[p] != REG_ENOTCONV && status[p] != REG_ELINESEARCH)
      worst = (reg_status)status[p];
  }
  if (s != REG_OK) return s;
  return worst;
}

reg_status reg_lockstep_matvec_time(reg_lockstep* L, int reps, double* ms) {
  if (!L || reps < 1 || !ms) return REG_EINVAL;
  return guarded(L, [&] {
    reg_lockstep::GraphEntry* e = nullptr;
    for (auto& g : L->graphs)
      if (g.in == L->wv && g.out == L->wo) e = &g;
    if (!e || !e->exec)
      fail(L, REG_ESTATE, "call reg_lockstep_hessian_matvec twice first (the graph is captured on "
                          "the second call)");
    set_mask(L, all_of(L->B));
    cudaEvent_t a, b;
    check(L, cudaEventCreate(&a), "event");
    check(L, cudaEventCreate(&b), "event");
    check(L, cudaEventRecord(a, L->st), "event");
    for (int r = 0; r < reps; ++r) {
      check(L, cudaGraphLaunch(e->exec, L->st), "graph launch");
      g_launch_count += e->kernels;
    }
    check(L, cudaEventRecord(b, L->st), "event");
    check(L, cudaEventSynchronize(b), "event");
    float t = 0.f;
    check(L, cudaEventElapsedTime(&t, a, b), "event");
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = (double)t / reps;
  });
}

reg_status reg_lockstep_info(const reg_lockstep* L, long long* points, int* tiles, int* launches) {
  if (!L) return REG_EINVAL;
  if (points) *points = L->NT;
  if (tiles) *tiles = L->ntiles;
  if (launches) {
    *launches = 0;
    for (const auto& g : L->graphs)
      if (g.in == L->kp && g.exec) *launches = (int)g.kernels;
  }
  return REG_OK;
}

const char* reg_lockstep_last_error(const reg_lockstep* L) { return L ? L->err.c_str() : "null batch"; }

}  // extern "C"
