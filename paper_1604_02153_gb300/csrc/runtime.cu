// Host runtime of libregnk: context and workspace management, the
// objective / gradient / Gauss-Newton Hessian pipelines, the Krylov solvers,
// the preconditioners and the inexact Newton loop, behind the C ABI of
// include/reg.h. All field arithmetic runs in the kernels of fft.cu,
// transport.cu and reduce.cu; the host only sequences launches and reads the
// FP64 scalars that steer the iterations.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <functional>
#include <initializer_list>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "reg.h"

using namespace regnk;

namespace regnk {
std::atomic<long long> g_launch_count{0};
thread_local int t_programmatic_launch = 1;
thread_local int t_graph_pdl = 0;
thread_local int t_level = 0;
thread_local int t_plain_fp32_reduce = 0;
}

namespace {

constexpr int kSpecSlots = 8;    // spectra in the FFT workspace of a level
constexpr int kScalars = 32;     // FP64 device scalar slots

enum Slot { S_A = 0, S_B, S_C, S_D, S_E, S_GINF, S_G2, S_J1, S_J2, S_DX, S_DY,
            S_PCG_OUTER = 16, S_PCG_INNER = 24 };
// offsets of the PCG scalars inside a PCG slot block
enum PcgSlot { P_RZ = 0, P_RZNEW, P_PQ, P_RR, P_BB };

struct Level {
  GridDims g;
  int nt = 0;
  float ht = 0.f;
  double h1 = 0, h2 = 0;
  float2* tw1 = nullptr;   // twiddles for length n1
  float2* tw2 = nullptr;   // twiddles for length n2
  float* mR = nullptr;
  float* mT = nullptr;
  float* v = nullptr;       // cached velocity (2N)
  float* cv = nullptr;      // its interpolation coefficients (2N)
  float* dX = nullptr;      // departure displacement, forward characteristic (2N)
  float* dY = nullptr;      // backward characteristic (2N)
  float* delta = nullptr;   // div v (N)
  float* delta_bar = nullptr;  // div v at Y_D (N)
  float* m = nullptr;       // state history m_0..m_nt ((nt+1) N)
  float* gm = nullptr;      // grad m_0..grad m_nt (2 (nt+1) N)
  float* G = nullptr;       // grad m_{j-1}(X_D), j = 1..nt (2 nt N)
  float* coef = nullptr;    // interpolation coefficients of one scalar field (N)
  float* tmp = nullptr;     // prefilter intermediate (2N)
  float* fA = nullptr;      // scalar ping-pong (N)
  float* fB = nullptr;
  float* c2 = nullptr;      // coefficients of a vector field (2N)
  float* vtD = nullptr;     // v~ at X_D (2N)
  float* b = nullptr;       // time-integral accumulator (2N)
  float* Av = nullptr;      // beta A v (2N)
  float* w1 = nullptr;      // vector scratch (2N)
  float* w2 = nullptr;      // vector scratch (2N)
  float2* spec = nullptr;   // kSpecSlots spectra
  bool have_images = false;
  bool have_v = false;      // v, dX, state valid
  bool have_gm = false;     // grad history valid for v
  bool have_div = false;    // delta, delta_bar, dY valid for v
  bool have_G = false;      // G valid for v
  int fuse_w = 0;           // box width of the fused prefilter+step kernels for v (0: off)
  bool lagrange = false;    // interpolation model of this level (cubic Lagrange or spline)
  int tile_adj = kDefaultStepTile;   // tile shapes of k_adjoint_step and k_incstate_step
  int tile_inc = kDefaultStepTile;
  // full-Newton matvec (problem grid only): adjoint history lambda_0..lambda_nt of
  // the last gradient, incremental state history, div(lambda_j v~), grad m~_j
  float* lam_hist = nullptr;  // (nt+1) N
  float* mt_hist = nullptr;   // (nt+1) N
  float* src = nullptr;       // (nt+1) N
  float* gmt = nullptr;       // 2 nt N
  float* prod = nullptr;      // 2 (nt+1) N
  bool have_lam = false;      // lam_hist belongs to the cached velocity
  // GN data term in one launch with tile-to-tile synchronisation (flow.cu):
  // cubic Lagrange levels with nt >= 2 whose tiles all fit the GPU at once
  bool flow = false;
  int flow_tx = 0, flow_ty = 0;     // tiles per axis
  unsigned* flow_flags = nullptr;   // one per tile
  double* flow_dmax = nullptr;      // largest |X_D - x|, |Y_D - x| in cells (2, device)
};

}  // namespace

struct reg_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  reg_options opt;
  double beta = 0;
  int nt = 0;
  bool two_level = false;
  bool incompressible = false;   // K = Leray projection (w = 0) instead of K = I
  bool full_newton = false;      // full Hessian on the problem grid (P_2L's coarse stays GN)
  double beta_w = 0;             // near-incompressible: weight of ||div v||^2_H1 (0: off;
                                 // then K is the multiplier of has_K below)
  float* rk2a = nullptr;         // RK2A comparator workspace (9 N), allocated on first use
  float* defmap = nullptr;       // deformation map workspace (10 N), allocated on first use
  Level fine, coarse;
  std::vector<void*> allocs;
  std::vector<std::pair<int, float2*>> tw;   // twiddle tables by length
  double* dsc = nullptr;          // device FP64 scalars
  double* hsc = nullptr;          // pinned host mirror
  double* partial = nullptr;      // reduction partials
  float* partialf = nullptr;
  int* dflag = nullptr;
  int* hflag = nullptr;
  // fine Krylov vectors (2N each)
  float *kx = nullptr, *kr = nullptr, *kz = nullptr, *kp = nullptr, *kq = nullptr;
  float *vtrial = nullptr, *gcur = nullptr, *vt_tmp = nullptr;
  // coarse vectors (2 Nc each)
  float *cx = nullptr, *cr = nullptr, *cd = nullptr, *cAd = nullptr, *crhs = nullptr,
        *cu = nullptr, *cq = nullptr, *cz = nullptr, *cp = nullptr;
  bool have_eig = false;
  double emin = 0, emax = 0, eig_beta = 0;
  bool have_gref = false;
  double gref_inf = 0, gref_2 = 0;
  double J_zero = 0;               // J(0), computed with the reference gradient
  double eta = 0.5;
  int coarse_matvecs = 0;
  std::string err;
  // per-kernel-class device time (diagnostics, reg_profile_*)
  bool prof = false;
  std::vector<cudaEvent_t> evpool;
  struct Rec { int cls; int level; cudaEvent_t a, b; double bytes; };
  std::vector<Rec> recs;
  // [level][class]: level 0 = the problem grid, 1 = the coarse grid of P_2L
  double prof_ms[2][REG_KC_COUNT] = {};
  double prof_bytes[2][REG_KC_COUNT] = {};
  long long prof_n[2][REG_KC_COUNT] = {};
  int cur_level = 0;
  // CUDA graphs of fixed launch sequences (fine matvec, P_2L with CHEB)
  cudaStream_t cap = nullptr;
  cudaStream_t side = nullptr;   // second stream for independent work (on_side)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool graphs = true;
  struct GraphEntry {
    std::string key;
    cudaGraphExec_t exec;
    long long kernels;
    std::vector<Rec> prof_recs;   // event pairs recorded inside the graph (profiling)
  };
  bool capturing = false;
  // persistent matvec: barrier state (2 unsigned) and error flag, device
  bool persistent = true;
  bool any_flow = false;         // a level runs the flow kernel (its waits share barerr)
  unsigned* bar = nullptr;
  int* barerr = nullptr;
  int* hbarerr = nullptr;
  std::vector<GraphEntry> graph_cache;
  double graph_beta = -1, graph_emin = -1, graph_emax = -1;
};

namespace {

struct CudaError {
  reg_status s;
};

void fail(reg_ctx* c, reg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  c->err = buf;
  throw CudaError{s};
}

void check(reg_ctx* c, cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(c, REG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void check_launch(reg_ctx* c, const char* what) { check(c, cudaGetLastError(), what); }

cudaEvent_t take_event(reg_ctx* c) {
  if (c->evpool.empty()) {
    cudaEvent_t e;
    check(c, cudaEventCreate(&e), "cudaEventCreate");
    return e;
  }
  cudaEvent_t e = c->evpool.back();
  c->evpool.pop_back();
  return e;
}

// Folds recorded event pairs into the per-class totals (synchronises).
void harvest(reg_ctx* c) {
  if (c->recs.empty()) return;
  check(c, cudaStreamSynchronize(c->st), "profile sync");
  for (auto& r : c->recs) {
    float ms = 0.f;
    check(c, cudaEventElapsedTime(&ms, r.a, r.b), "cudaEventElapsedTime");
    c->prof_ms[r.level][r.cls] += ms;
    c->prof_bytes[r.level][r.cls] += r.bytes;
    c->prof_n[r.level][r.cls] += 1;
    c->evpool.push_back(r.a);
    c->evpool.push_back(r.b);
  }
  c->recs.clear();
}

// Brackets the launches of one kernel class with events when profiling is
// on; bytes = algorithmic bytes moved by those launches.
class Prof {
 public:
  Prof(reg_ctx* c, int cls, double bytes) : c_(c) {
    if (!c->prof) return;
    if (c->recs.size() >= 8192 && !c->capturing) harvest(c);
    r_.cls = cls;
    r_.level = c->cur_level;
    r_.bytes = bytes;
    r_.a = take_event(c);
    r_.b = take_event(c);
    record(r_.a);
  }
  ~Prof() {
    if (!c_->prof) return;
    record(r_.b);
    c_->recs.push_back(r_);
  }

 private:
  // inside a stream capture an event record only becomes a graph node with
  // the external flag
  void record(cudaEvent_t e) {
    if (c_->capturing)
      cudaEventRecordWithFlags(e, c_->st, cudaEventRecordExternal);
    else
      cudaEventRecord(e, c_->st);
  }

 public:

 private:
  reg_ctx* c_;
  reg_ctx::Rec r_{};
};

template <typename T>
T* dalloc(reg_ctx* c, size_t count) {
  void* p = nullptr;
  const cudaError_t e = cudaMalloc(&p, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
  if (e != cudaSuccess) fail(c, REG_ENOMEM, "cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
  c->allocs.push_back(p);
  return static_cast<T*>(p);
}

float2* twiddles(reg_ctx* c, int n) {
  for (auto& e : c->tw)
    if (e.first == n) return e.second;
  std::vector<float2> h(n);
  for (int m = 0; m < n; ++m) {
    const double a = -2.0 * M_PI * (double)m / (double)n;
    h[m] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  float2* d = dalloc<float2>(c, n);
  check(c, cudaMemcpy(d, h.data(), n * sizeof(float2), cudaMemcpyHostToDevice), "twiddle upload");
  c->tw.push_back({n, d});
  return d;
}

void alloc_level(reg_ctx* c, Level& L, int n1, int n2, int nt) {
  L.g = make_grid(n1, n2);
  L.nt = nt;
  L.ht = 1.0f / (float)nt;
  L.h1 = 2.0 * M_PI / n1;
  L.h2 = 2.0 * M_PI / n2;
  L.tw1 = twiddles(c, n1);
  L.tw2 = twiddles(c, n2);
  const size_t N = (size_t)L.g.N;
  L.mR = dalloc<float>(c, N);
  L.mT = dalloc<float>(c, N);
  L.v = dalloc<float>(c, 2 * N);
  L.cv = dalloc<float>(c, 2 * N);
  L.dX = dalloc<float>(c, 2 * N);
  L.dY = dalloc<float>(c, 2 * N);
  L.delta = dalloc<float>(c, N);
  L.delta_bar = dalloc<float>(c, N);
  L.m = dalloc<float>(c, (nt + 1) * N);
  L.gm = dalloc<float>(c, 2 * (nt + 1) * N);
  L.G = dalloc<float>(c, 2 * nt * N);
  L.coef = dalloc<float>(c, N);
  L.tmp = dalloc<float>(c, 2 * N);
  L.fA = dalloc<float>(c, N);
  L.fB = dalloc<float>(c, N);
  L.c2 = dalloc<float>(c, 2 * N);
  L.vtD = dalloc<float>(c, 2 * N);
  L.b = dalloc<float>(c, 2 * N);
  L.Av = dalloc<float>(c, 2 * N);
  L.w1 = dalloc<float>(c, 2 * N);
  L.w2 = dalloc<float>(c, 2 * N);
  L.spec = dalloc<float2>(c, kSpecSlots * (size_t)L.g.spec);
  // the flow kernel needs every tile's block resident at once
  const int tiles = flow_tiles(n1, n2);
  if (L.lagrange && nt >= 2 && c->opt.flow_matvec && !c->persistent && tiles > 0 &&
      flow_capacity(n1, n2) >= tiles) {
    L.flow = true;
    L.flow_tx = n1 / 32;
    L.flow_ty = tiles / L.flow_tx;
    L.flow_flags = dalloc<unsigned>(c, tiles);
    L.flow_dmax = dalloc<double>(c, 2);
    c->any_flow = true;
  }
}


// Attributes the launches inside its lifetime to a grid level (profiling).
class LevelScope {
 public:
  LevelScope(reg_ctx* c, const Level& L) : c_(c), prev_(c->cur_level) {
    c->cur_level = (&L == &c->coarse) ? 1 : 0;
    t_level = c->cur_level;
  }
  ~LevelScope() {
    c_->cur_level = prev_;
    t_level = prev_;
  }

 private:
  reg_ctx* c_;
  int prev_;
};

void drop_graphs(reg_ctx* c) {
  for (auto& g : c->graph_cache) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& r : g.prof_recs) {
      c->evpool.push_back(r.a);
      c->evpool.push_back(r.b);
    }
  }
  c->graph_cache.clear();
}

// Launch attribute of this context for the duration of one call (see
// launch_k); restored when the call returns.
struct LaunchModeScope {
  int saved;
  explicit LaunchModeScope(int mode) : saved(t_programmatic_launch) { t_programmatic_launch = mode; }
  ~LaunchModeScope() { t_programmatic_launch = saved; }
};

// Programmatic edges for the launches captured into a graph (see launch_k).
struct GraphPdlScope {
  int saved;
  explicit GraphPdlScope(int mode) : saved(t_graph_pdl) { t_graph_pdl = mode; }
  ~GraphPdlScope() { t_graph_pdl = saved; }
};

// Reduction precision of this context for the duration of one call.
struct ReducePrecisionScope {
  int saved;
  explicit ReducePrecisionScope(int plain) : saved(t_plain_fp32_reduce) { t_plain_fp32_reduce = plain; }
  ~ReducePrecisionScope() { t_plain_fp32_reduce = saved; }
};

// Tile shapes of the step kernels (k_adjoint_step, k_incstate_step) for a
// level. step_tile > 0 fixes the shape, 0 takes the default; -1 times every
// shape on this level's grid and keeps the fastest, once per (device, grid,
// interpolation model) in this process: later contexts (a batch of problems
// on the same grids) reuse the choice. The timing runs the middle step of
// each kernel on the level's own buffers, zeroed first (every stencil at its
// own node: the same loads and arithmetic as a solve, in the same pattern
// up to the displacement), eight launches at a time, best of three; the
// default shape is kept unless another one is more than 3 % faster.
std::mutex g_tile_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tiles;

void choose_step_tiles(reg_ctx* c, Level& L) {
  const int o = c->opt.step_tile;
  if (o >= 0) {
    L.tile_adj = L.tile_inc = (o > 0 ? o : kDefaultStepTile);
    return;
  }
  const auto key = std::make_tuple(c->device, L.g.n1, L.g.n2, (int)L.lagrange);
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    const auto it = g_tiles.find(key);
    if (it != g_tiles.end()) {
      L.tile_adj = it->second.first;
      L.tile_inc = it->second.second;
      return;
    }
  }
  const size_t N = (size_t)L.g.N;
  for (float* p : {L.coef, L.delta, L.delta_bar})
    check(c, cudaMemsetAsync(p, 0, N * sizeof(float), c->st), "memset");
  for (float* p : {L.dX, L.dY, L.gm, L.G, L.vtD, L.b, L.w1})
    check(c, cudaMemsetAsync(p, 0, 2 * N * sizeof(float), c->st), "memset");
  LaunchModeScope plain(0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  check(c, cudaEventCreate(&e0), "cudaEventCreate");
  const cudaError_t ee = cudaEventCreate(&e1);
  if (ee != cudaSuccess) cudaEventDestroy(e0);
  check(c, ee, "cudaEventCreate");
  const int n1 = L.g.n1, n2 = L.g.n2, lg = L.lagrange ? 1 : 0;
  const float ht = L.ht;
  auto best_ms = [&](const std::function<void()>& launch) {
    launch();
    launch();
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, c->st);
      for (int r = 0; r < 8; ++r) launch();
      cudaEventRecord(e1, c->st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        break;
      best = std::fmin(best, ms);
    }
    return best;
  };
  float t_adj[kStepTiles + 1], t_inc[kStepTiles + 1];
  for (int k = 1; k <= kStepTiles; ++k) {
    t_adj[k] = best_ms([&] {
      launch_adjoint_step(k, n1, n2, ht, ht, L.coef, L.dY, L.delta, L.delta_bar, L.gm, L.fA, L.b,
                          lg, c->st);
    });
    t_inc[k] = best_ms([&] {
      launch_incstate_step(k, n1, n2, ht, L.coef, L.dX, L.w1, L.vtD, L.G, L.gm, L.fB, 0, lg, c->st);
    });
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check(c, e, "step tile timing");
  auto pick_best = [](const float* t) {
    int b = kDefaultStepTile;
    for (int k = 1; k <= kStepTiles; ++k)
      if (t[k] < t[b]) b = k;
    return (t[b] < 0.97f * t[kDefaultStepTile]) ? b : kDefaultStepTile;
  };
  L.tile_adj = pick_best(t_adj);
  L.tile_inc = pick_best(t_inc);
  std::lock_guard<std::mutex> lk(g_tile_mu);
  g_tiles[key] = {L.tile_adj, L.tile_inc};
}

// Runs `body` (a fixed sequence of launches on c->st, no host synchronisation)
// as a CUDA graph: the first call of a key runs eagerly, the second captures
// the sequence on a private stream, later calls replay it on c->st. Graphs
// are dropped when beta or the Chebyshev bounds change (they are launch
// arguments). While profiling, separate graphs are captured whose kernels
// are bracketed by event-record nodes; after each replay the stream is
// synchronised and those events are read, so kernel times carry no host
// launch gaps. Returns true when the body ran eagerly (host-side counters
// inside it ran).
template <typename Body>
bool graphed(reg_ctx* c, const std::string& key0, Body body) {
  if (!c->graphs) {
    body();
    return true;
  }
  const std::string key = c->prof ? "P" + key0 : key0;
  if (c->graph_beta != c->beta || c->graph_emin != c->emin || c->graph_emax != c->emax) {
    drop_graphs(c);
    c->graph_beta = c->beta;
    c->graph_emin = c->emin;
    c->graph_emax = c->emax;
  }
  reg_ctx::GraphEntry* e = nullptr;
  for (auto& g : c->graph_cache)
    if (g.key == key) e = &g;
  if (!e) {
    c->graph_cache.push_back({key, nullptr, 0, {}});
    body();
    return true;
  }
  if (!e->exec) {
    cudaStream_t user = c->st;
    const size_t rec0 = c->recs.size();
    check(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    c->st = c->cap;
    c->capturing = true;
    cudaGraph_t graph = nullptr;
    try {
      // plain launches inside graphs, unless reg_options.graph_pdl asks for
      // programmatic edges on the coarse grid (1) or everywhere (2)
      LaunchModeScope plain(0);
      GraphPdlScope gp(c->opt.graph_pdl);
      body();
    } catch (...) {
      // capture failed (e.g. a launch form the graph cannot hold): drop the
      // capture, stop using graphs in this context and run eagerly
      cudaStreamEndCapture(c->cap, &graph);
      if (graph) cudaGraphDestroy(graph);
      c->st = user;
      c->capturing = false;
      c->recs.resize(rec0);
      cudaGetLastError();
      c->graphs = false;
      drop_graphs(c);
      body();
      return true;
    }
    c->st = user;
    c->capturing = false;
    check(c, cudaStreamEndCapture(c->cap, &graph), "end capture");
    // event pairs recorded during capture belong to the graph
    e->prof_recs.assign(c->recs.begin() + rec0, c->recs.end());
    c->recs.resize(rec0);
    // the captured launches were counted; count them once per replay instead
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
    check(c, ie, "graph instantiate");
  }
  check(c, cudaGraphLaunch(e->exec, c->st), "graph launch");
  g_launch_count += e->kernels;
  if (!e->prof_recs.empty()) {
    check(c, cudaStreamSynchronize(c->st), "profile sync");
    for (auto& r : e->prof_recs) {
      float ms = 0.f;
      check(c, cudaEventElapsedTime(&ms, r.a, r.b), "cudaEventElapsedTime");
      c->prof_ms[r.level][r.cls] += ms;
      c->prof_bytes[r.level][r.cls] += r.bytes;
      c->prof_n[r.level][r.cls] += 1;
    }
  }
  return false;
}

// the key names the buffers and the fused-kernel box widths of both levels
// (a launch sequence recorded for one width must not replay for another)
std::string graph_key(const reg_ctx* c, const char* what, const void* a, const void* b) {
  char buf[128];
  snprintf(buf, sizeof buf, "%s:%p:%p:%d:%d", what, a, b, c->fine.fuse_w, c->coarse.fuse_w);
  return buf;
}

// Runs `body` (launches on c->st) on the side stream after everything
// queued on c->st so far; join_side() makes c->st wait for it. Works eagerly
// and under stream capture (the fork and join become graph edges).
template <typename Body>
void on_side(reg_ctx* c, Body body) {
  check(c, cudaEventRecord(c->ev_fork, c->st), "fork");
  check(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork");
  cudaStream_t main = c->st;
  c->st = c->side;
  body();
  c->st = main;
  check(c, cudaEventRecord(c->ev_join, c->side), "join");
}

void join_side(reg_ctx* c) { check(c, cudaStreamWaitEvent(c->st, c->ev_join, 0), "join"); }

// ---------------------------------------------------------------------------
// spectral operators

ColArgs col_args(const Level& L, int op, double beta, int p, double s, double beta_w = 0.0) {
  ColArgs a{};
  a.beta_w = (float)beta_w;
  a.n1_in = a.n1_out = a.n1 = L.g.n1;
  a.n2_in = a.n2_out = a.n2 = L.g.n2;
  a.nk1_out = L.g.nk1;
  a.op = op;
  a.beta = (float)beta;
  a.p = p;
  a.s = (float)s;
  a.scale = (float)(1.0 / (double)L.g.N);
  a.tw_in = a.tw_out = L.tw2;
  return a;
}

// out (groups*fout fields) = op(in (groups*fin fields)) [+ add], on level L.
// With `cheb`, the inverse row pass ends in one Chebyshev iteration on its
// output instead of storing it (see ChebEpilogue).
void spectral(reg_ctx* c, Level& L, int op, double s, const float* in, int fin, int groups,
              float* out, int fout, const float* add, const ChebEpilogue* cheb = nullptr) {
  LevelScope ls(c, L);
  const GridDims& g = L.g;
  const int per = fin + fout;
  const int chunk = kSpecSlots / per;
  for (int g0 = 0; g0 < groups; g0 += chunk) {
    const int ng = groups - g0 < chunk ? groups - g0 : chunk;
    float2* sin = L.spec;
    float2* sout = L.spec + (size_t)ng * fin * g.spec;
    {
      Prof P(c, REG_KC_FFT_ROWS, (double)ng * fin * (4.0 * g.N + 8.0 * g.spec));
      fft_rows_r2c(g.n1, g.n2, in + (size_t)g0 * fin * g.N, g.N, sin, g.spec, ng * fin, L.tw1, c->st);
    }
    ColArgs a = col_args(L, op, c->beta, c->opt.reg_norm, s, c->beta_w);
    a.in = sin;
    a.in_fstride = g.spec;
    a.out = sout;
    a.out_fstride = g.spec;
    a.nin = fin;
    a.nout = fout;
    {
      Prof P(c, REG_KC_FFT_COLS, (double)ng * (fin + fout) * 8.0 * g.spec);
      fft_cols(a, ng, c->st);
    }
    {
      Prof P(c, REG_KC_FFT_ROWS, (double)ng * fout * (8.0 * g.spec + (add ? 8.0 : 4.0) * g.N));
      ChebEpilogue ce;
      if (cheb) {
        ce = *cheb;
        ce.r += (size_t)g0 * fout * g.N;
        ce.d += (size_t)g0 * fout * g.N;
        ce.x += (size_t)g0 * fout * g.N;
      }
      fft_rows_c2r(g.n1, g.n2, sout, g.spec, out + (size_t)g0 * fout * g.N, g.N,
                   add ? add + (size_t)g0 * fout * g.N : nullptr, g.N, ng * fout, L.tw1, c->st,
                   cheb ? &ce : nullptr);
    }
  }
  check_launch(c, "spectral operator");
}

// spectral() split in two for a single chunk (groups * (fin + fout) <=
// kSpecSlots), so that independent work can run between the halves:
// spectral_fwd leaves the output spectra in L.spec, spectral_inv transforms
// them back (with the addend).
void spectral_fwd(reg_ctx* c, Level& L, int op, double s, const float* in, int fin, int groups,
                  int fout) {
  LevelScope ls(c, L);
  const GridDims& g = L.g;
  float2* sin = L.spec;
  float2* sout = L.spec + (size_t)groups * fin * g.spec;
  {
    Prof P(c, REG_KC_FFT_ROWS, (double)groups * fin * (4.0 * g.N + 8.0 * g.spec));
    fft_rows_r2c(g.n1, g.n2, in, g.N, sin, g.spec, groups * fin, L.tw1, c->st);
  }
  ColArgs a = col_args(L, op, c->beta, c->opt.reg_norm, s, c->beta_w);
  a.in = sin;
  a.in_fstride = g.spec;
  a.out = sout;
  a.out_fstride = g.spec;
  a.nin = fin;
  a.nout = fout;
  {
    Prof P(c, REG_KC_FFT_COLS, (double)groups * (fin + fout) * 8.0 * g.spec);
    fft_cols(a, groups, c->st);
  }
  check_launch(c, "spectral operator");
}

void spectral_inv(reg_ctx* c, Level& L, int fin, int groups, float* out, int fout,
                  const float* add) {
  LevelScope ls(c, L);
  const GridDims& g = L.g;
  float2* sout = L.spec + (size_t)groups * fin * g.spec;
  {
    Prof P(c, REG_KC_FFT_ROWS, (double)groups * fout * (8.0 * g.spec + (add ? 8.0 : 4.0) * g.N));
    fft_rows_c2r(g.n1, g.n2, sout, g.spec, out, g.N, add, g.N, groups * fout, L.tw1, c->st);
  }
  check_launch(c, "spectral operator");
}

// Spectral resampling of F fields from level A to level B (restriction or
// prolongation) with multiplier op(s), plus an optional addend on B.
void resample(reg_ctx* c, Level& A, Level& B, int op, double s, const float* in, int F,
              float* out, const float* add) {
  LevelScope ls(c, A);
  float2* sin = c->fine.spec;
  float2* sout = c->fine.spec + (size_t)F * A.g.spec;
  {
    Prof P(c, REG_KC_FFT_ROWS, (double)F * (4.0 * A.g.N + 8.0 * A.g.spec));
    fft_rows_r2c(A.g.n1, A.g.n2, in, A.g.N, sin, A.g.spec, F, A.tw1, c->st);
  }
  ColArgs a = col_args(A, op, c->beta, c->opt.reg_norm, s, c->beta_w);
  a.in = sin;
  a.in_fstride = A.g.spec;
  a.out = sout;
  a.out_fstride = B.g.spec;
  a.nin = 1;
  a.nout = 1;
  a.n1_out = B.g.n1;
  a.n2_out = B.g.n2;
  a.nk1_out = B.g.nk1;
  a.tw_out = B.tw2;
  {
    Prof P(c, REG_KC_FFT_COLS, (double)F * 8.0 * (A.g.spec + B.g.spec));
    fft_cols(a, F, c->st);
  }
  {
    Prof P(c, REG_KC_FFT_ROWS, (double)F * (8.0 * B.g.spec + (add ? 8.0 : 4.0) * B.g.N));
    fft_rows_c2r(B.g.n1, B.g.n2, sout, B.g.spec, out, B.g.N, add, B.g.N, F, B.tw1, c->st);
  }
  check_launch(c, "spectral resampling");
}

// Spectral resampling of F fields between square grids of n_a and n_b =
// n_a / 2 or 2 n_a points per axis (same truncation / zero padding as
// resample(), for grids that are not levels of the context).
void resample_square(reg_ctx* c, int na, int nb, const float* in, int F, float* out) {
  const GridDims A = make_grid(na, na), B = make_grid(nb, nb);
  float2* sin = c->fine.spec;
  float2* sout = c->fine.spec + (size_t)F * A.spec;
  fft_rows_r2c(na, na, in, A.N, sin, A.spec, F, twiddles(c, na), c->st);
  ColArgs a{};
  a.n1_in = a.n1 = na;
  a.n2_in = a.n2 = na;
  a.n1_out = nb;
  a.n2_out = nb;
  a.nk1_out = B.nk1;
  a.op = SPOP_SCALE;
  a.beta = 1.f;
  a.p = 1;
  a.s = 0.f;
  a.scale = (float)(1.0 / (double)A.N);
  a.tw_in = twiddles(c, na);
  a.tw_out = twiddles(c, nb);
  a.in = sin;
  a.in_fstride = A.spec;
  a.out = sout;
  a.out_fstride = B.spec;
  a.nin = 1;
  a.nout = 1;
  fft_cols(a, F, c->st);
  fft_rows_c2r(nb, nb, sout, B.spec, out, B.N, nullptr, B.N, F, twiddles(c, nb), c->st);
  check_launch(c, "spectral resampling");
}

// The operator K of the reduced gradient and the Hessian (eq. control-elim,
// eq. hessian-matvec): the identity (compressible), the Leray projection
// (incompressible, w = 0, §3.1) or, for the near-incompressible problem, the
// 2 -> 2 multiplier I - c(k) kd kd^T / |kd|^2 with
// c = beta_w (1 + |k|^2) |kd|^2 / (beta |k|^2p + beta_w (1 + |k|^2) |kd|^2)
// that eliminating the mass source w = div v and its multiplier p from the
// control equations of Appendix A leaves (beta A M^-1, M = beta A -
// beta_w grad (I - Lap) div); and K times (beta A)^s for P_2L's coarse
// operator.
bool has_K(const reg_ctx* c) { return c->incompressible || c->beta_w > 0.0; }
int K_op(const reg_ctx* c) { return c->incompressible ? SPOP_LERAY : SPOP_KW; }
int regpow_K_op(const reg_ctx* c) { return c->incompressible ? SPOP_REGPOW_LERAY : SPOP_REGPOW_KW; }

// interpolation coefficients of F consecutive fields (prefilter for the
// spline model; the samples themselves for Lagrange)
const float* coefficients(reg_ctx* c, Level& L, const float* u, int F, float* dst) {
  LevelScope ls(c, L);
  if (L.lagrange) return u;
  Prof P(c, REG_KC_PREFILTER, 16.0 * F * L.g.N);
  for (int f = 0; f < F; ++f)
    launch_prefilter(L.g.n1, L.g.n2, u + (size_t)f * L.g.N, L.tmp, dst + (size_t)f * L.g.N, 1, c->st);
  check_launch(c, "prefilter");
  return dst;
}

// ---------------------------------------------------------------------------
// scalars

double* slot(reg_ctx* c, int s) { return c->dsc + s; }

void read_slots(reg_ctx* c, int first, int count) {
  check(c, cudaMemcpyAsync(c->hsc + first, c->dsc + first, count * sizeof(double),
                           cudaMemcpyDeviceToHost, c->st), "scalar read");
  // only the persistent matvec and the flow kernel can raise the wait flag
  const bool waits = c->persistent || c->any_flow;
  if (waits)
    check(c, cudaMemcpyAsync(c->hbarerr, c->barerr, sizeof(int), cudaMemcpyDeviceToHost, c->st),
          "barrier flag read");
  check(c, cudaStreamSynchronize(c->st), "stream synchronize");
  if (waits && *c->hbarerr) {
    // a persistent or flow kernel gave up a bounded wait: reset the state
    cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), c->st);
    cudaMemsetAsync(c->barerr, 0, sizeof(int), c->st);
    cudaStreamSynchronize(c->st);
    *c->hbarerr = 0;
    fail(c, REG_ETIMEOUT, c->persistent
                              ? "grid barrier wait of the persistent matvec timed out"
                              : "tile wait of the flow matvec timed out");
  }
}

void dot_async(reg_ctx* c, const float* a, const float* b, long long n, int s) {
  Prof P(c, REG_KC_REDUCE, 8.0 * n);
  launch_dot(a, b, n, c->partial, slot(c, s), c->st);
}

double dot_sync(reg_ctx* c, const float* a, const float* b, long long n, int s) {
  dot_async(c, a, b, n, s);
  check_launch(c, "dot");
  read_slots(c, s, 1);
  return c->hsc[s];
}

// ---------------------------------------------------------------------------
// level pipelines

// Caches v, its characteristics and the state history m_0..m_nt (§3.3.2).
void set_velocity(reg_ctx* c, Level& L, const float* v) {
  LevelScope ls(c, L);
  const GridDims& g = L.g;
  const size_t N = (size_t)g.N;
  if (v != L.v) check(c, cudaMemcpyAsync(L.v, v, 2 * N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy v");
  const float* cv = coefficients(c, L, L.v, 2, L.cv);
  {
    Prof P(c, REG_KC_DEPARTURE, 32.0 * N);
    launch_departure(g.n1, g.n2, L.ht, L.v, cv, L.dX, L.dY, L.lagrange, c->st);
  }
  // largest displacement component (cells): decides whether the fused
  // prefilter+step kernels' coefficient box covers every stencil
  L.fuse_w = 0;
  if (!L.lagrange && c->opt.fused_transport) {
    {
      Prof P(c, REG_KC_REDUCE, 16.0 * N);
      launch_maxabs(L.dX, 2 * (long long)N, c->partialf, slot(c, S_DX), c->st);
      launch_maxabs(L.dY, 2 * (long long)N, c->partialf, slot(c, S_DY), c->st);
    }
    read_slots(c, S_DX, 2);
    L.fuse_w = fused_box_width(std::fmax(c->hsc[S_DX], c->hsc[S_DY]));
  }
  if (L.flow) {   // the flow kernel reads its tiles' reach from these (no host sync)
    Prof P(c, REG_KC_REDUCE, 16.0 * N);
    launch_maxabs(L.dX, 2 * (long long)N, c->partialf, L.flow_dmax, c->st);
    launch_maxabs(L.dY, 2 * (long long)N, c->partialf, L.flow_dmax + 1, c->st);
  }
  check(c, cudaMemcpyAsync(L.m, L.mT, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy m_T");
  for (int j = 1; j <= L.nt; ++j) {
    if (L.fuse_w) {   // prefilter of m_{j-1} inside the gather
      Prof P(c, REG_KC_GATHER, 16.0 * N);
      launch_gather_fused(L.fuse_w, g.n1, g.n2, L.m + (j - 1) * N, 0, 1, L.dX, L.m + j * N, c->st);
      continue;
    }
    const float* cm = coefficients(c, L, L.m + (j - 1) * N, 1, L.coef);
    {
      Prof P(c, REG_KC_GATHER, 16.0 * N);
      launch_state_step(g.n1, g.n2, cm, L.dX, L.m + j * N, L.lagrange, c->st);
    }
  }
  check_launch(c, "state solve");
  L.have_v = true;
  L.have_lam = false;
  L.have_gm = false;
  L.have_div = true;   // dY computed together with dX; delta below
  L.have_G = false;
  // div v and div v at Y_D
  spectral(c, L, SPOP_DIV, 0.0, L.v, 2, 1, L.delta, 1, nullptr);
  if (L.fuse_w) {
    Prof P(c, REG_KC_GATHER, 16.0 * N);
    launch_gather_fused(L.fuse_w, g.n1, g.n2, L.delta, 0, 1, L.dY, L.delta_bar, c->st);
  } else {
    const float* cd = coefficients(c, L, L.delta, 1, L.coef);
    Prof P(c, REG_KC_GATHER, 16.0 * N);
    launch_gather(g.n1, g.n2, cd, L.dY, L.delta_bar, 1, 0, L.lagrange, c->st);
  }
  check_launch(c, "div v");
}

void ensure_grad_history(reg_ctx* c, Level& L) {
  if (L.have_gm) return;
  const size_t N = (size_t)L.g.N;
  // grad m_1..grad m_nt (grad m_0 = grad m_T is set with the images)
  spectral(c, L, SPOP_GRAD, 0.0, L.m + N, 1, L.nt, L.gm + 2 * N, 2, nullptr);
  L.have_gm = true;
}

void ensure_G(reg_ctx* c, Level& L) {
  LevelScope ls(c, L);
  if (L.have_G) return;
  ensure_grad_history(c, L);
  const size_t N = (size_t)L.g.N;
  for (int j = 1; j <= L.nt; ++j) {
    if (L.fuse_w) {
      Prof P(c, REG_KC_GATHER, 24.0 * N);
      launch_gather_fused(L.fuse_w, L.g.n1, L.g.n2, L.gm + 2 * (j - 1) * N, (long long)N, 2, L.dX,
                          L.G + 2 * (j - 1) * N, c->st);
      continue;
    }
    const float* cg = coefficients(c, L, L.gm + 2 * (j - 1) * N, 2, L.c2);
    {
      Prof P(c, REG_KC_GATHER, 24.0 * N);
      launch_gather(L.g.n1, L.g.n2, cg, L.dX, L.G + 2 * (j - 1) * N, 2, (long long)N, L.lagrange, c->st);
    }
  }
  check_launch(c, "G history");
  L.have_G = true;
}

// J = 1/2 <m_1 - m_R, m_1 - m_R>_h + beta/2 <v, A v>_h (eq. varopt:objective);
// leaves beta A v in L.Av.
double objective(reg_ctx* c, Level& L) {
  LevelScope ls(c, L);
  const size_t N = (size_t)L.g.N;
  spectral(c, L, SPOP_REGPOW, 1.0, L.v, 1, 2, L.Av, 1, nullptr);
  // near-incompressible: the regularisation of J is beta/2 <v, A v> +
  // beta_w/2 ||div v||^2_H1 = 1/2 <v, R v> (R the 2 -> 2 multiplier
  // beta A - beta_w grad (I - Lap) div); the gradient keeps beta A v
  const float* Rv = L.Av;
  if (c->beta_w > 0.0) {
    spectral(c, L, SPOP_REGW, 1.0, L.v, 2, 1, L.w1, 2, nullptr);
    Rv = L.w1;
  }
  {
    Prof P(c, REG_KC_REDUCE, 8.0 * N);
    launch_sumsq_diff(L.m + L.nt * N, L.mR, (long long)N, c->partial, slot(c, S_J1), c->st);
  }
  {
    Prof P(c, REG_KC_REDUCE, 16.0 * N);
    launch_dot(L.v, Rv, 2 * (long long)N, c->partial, slot(c, S_J2), c->st);
  }
  check_launch(c, "objective");
  read_slots(c, S_J1, 2);
  const double hh = L.h1 * L.h2;
  return 0.5 * hh * c->hsc[S_J1] + 0.5 * hh * c->hsc[S_J2];
}

// Algorithmic bytes per grid point of the transport steps, as the
// profile counts them (each field the step needs read once, each result
// written once): an incremental state step moves m~_{j-1} in, m~_j out and
// the two time-level fields G_j, grad m_j (24 B); the first also reads v~
// and X_D, the matvec's per-velocity inputs (+16); the last also hands over
// b~ (+8). An adjoint step moves lambda_{j+1} in, lambda_j out and grad m_j
// (16 B); the first also reads Y_D, div v and div v(Y_D) (+16). The
// kernels move more (the running sum b, v~(X_D) and v~ at every step):
// those re-reads are the kernels' cost, not the method's.
double kIncStepBytes(int j, int nt) { return 24.0 + (j == 1 ? 16.0 : 0.0) + (j == nt ? 8.0 : 0.0); }
double kAdjStepBytes(bool first) { return 16.0 + (first ? 16.0 : 0.0); }

// One fused adjoint step (prefilter of lambda_{j+1} inside the step) and one
// fused incremental state step j >= 2 (b non-NULL for the last, j = nt,
// where gmj is grad m_nt).
void adjoint_fused(reg_ctx* c, Level& L, float wb, const float* lam_next, const float* gmj,
                   float* lam_out, float* b) {
  launch_adjoint_fused(L.fuse_w, L.g.n1, L.g.n2, L.ht, wb, lam_next, L.dY, L.delta, L.delta_bar,
                       gmj, lam_out, b, c->st);
}

void incstate_fused(reg_ctx* c, Level& L, const float* m_prev, const float* vt, const float* Gj,
                    const float* gmj, float* out, float* b) {
  launch_incstate_fused(L.fuse_w, L.g.n1, L.g.n2, L.ht, m_prev, L.dX, vt, L.vtD, Gj, gmj, out,
                        b ? gmj : nullptr, b, c->st);
}

// b = int_0^1 lambda grad m dt by the adjoint solve (eq. adj-slm), trapezoid in
// time; g = beta A v + b. Needs objective() for L.Av.
void gradient(reg_ctx* c, Level& L, float* g_out) {
  LevelScope ls(c, L);
  ensure_grad_history(c, L);
  const GridDims& gd = L.g;
  const size_t N = (size_t)gd.N;
  const int nt = L.nt;
  const float ht = L.ht;
  // the full-Newton matvec needs every lambda_j: then they are kept in lam_hist
  float* hist = L.lam_hist;
  float* lam = hist ? hist + nt * N : L.fA;
  float* lam2 = L.fB;
  {
    Prof P(c, REG_KC_VECTOR, 28.0 * N);
    launch_adjoint_init(gd.n1, gd.n2, 0.5f * ht, L.mR, L.m + nt * N, L.gm + 2 * nt * N, lam, L.b, 1.f, c->st);
  }
  for (int j = nt - 1; j >= 0; --j) {
    const float wb = ht * (j == 0 ? 0.5f : 1.0f);
    if (hist) lam2 = hist + j * N;
    if (L.fuse_w) {   // prefilter of lambda_{j+1} inside the step
      Prof P(c, REG_KC_ADJOINT_STEP, kAdjStepBytes(j == nt - 1) * N);
      adjoint_fused(c, L, wb, lam, L.gm + 2 * j * N, lam2, L.b);
      std::swap(lam, lam2);
      continue;
    }
    const float* cl = coefficients(c, L, lam, 1, L.coef);
    {
      Prof P(c, REG_KC_ADJOINT_STEP, kAdjStepBytes(j == nt - 1) * N);
      launch_adjoint_step(L.tile_adj, gd.n1, gd.n2, ht, wb, cl, L.dY, L.delta, L.delta_bar,
                          L.gm + 2 * j * N, lam2, L.b, L.lagrange, c->st);
    }
    std::swap(lam, lam2);
  }
  check_launch(c, "adjoint solve");
  if (hist) L.have_lam = true;
  if (has_K(c)) {   // g = beta A v + K[b]
    spectral(c, L, K_op(c), 0.0, L.b, 2, 1, g_out, 2, L.Av);
  } else {
    Prof P(c, REG_KC_VECTOR, 24.0 * N);
    launch_lincomb(2 * (long long)N, 1.f, L.Av, 1.f, L.b, g_out, c->st);
  }
  check_launch(c, "gradient");
}

// beta A v~ + K[b~] with K the Leray projection (incompressible) or the
// near-incompressible K, with b~ in L.b; L.w1 holds beta A v~ in between.
void finish_hessian_K(reg_ctx* c, Level& L, const float* vt, float* out) {
  spectral(c, L, SPOP_REGPOW, 1.0, vt, 1, 2, L.w1, 1, nullptr);
  spectral(c, L, K_op(c), 0.0, L.b, 2, 1, out, 2, L.w1);
}

// Gauss-Newton Hessian matvec (eq. hessian-matvec, GN); data_only drops beta A vt.
void hessian_core(reg_ctx* c, Level& L, const float* vt, float* out, bool data_only);

void hessian(reg_ctx* c, Level& L, const float* vt, float* out, bool data_only) {
  ensure_G(c, L);
  hessian_core(c, L, vt, out, data_only);
}

// one cooperative launch for the data term b~ (matvec.cu)
void data_term_persistent(reg_ctx* c, Level& L, const float* vt, float* b) {
  LevelScope ls(c, L);
  MatvecArgs a{};
  a.n1 = L.g.n1;
  a.n2 = L.g.n2;
  a.log1 = L.g.log1;
  a.nt = L.nt;
  a.lagrange = L.lagrange;
  a.N = L.g.N;
  a.ht = L.ht;
  a.vt = vt;
  a.dX = L.dX;
  a.dY = L.dY;
  a.delta = L.delta;
  a.delta_bar = L.delta_bar;
  a.gm = L.gm;
  a.G = L.G;
  a.c2 = L.c2;
  a.vtD = L.vtD;
  a.fA = L.fA;
  a.fB = L.fB;
  a.coef = L.coef;
  a.b = b;
  a.bar = c->bar;
  a.err = c->barerr;
  a.missing = c->opt.inject_barrier_timeout ? 1u : 0u;
  // algorithmic bytes per point: v~(X_D) and the first step 52, each later
  // incremental state step 48, each incremental adjoint step 48, each of the
  // 2 nt + 1 prefilters 8 (spline only)
  const double per_point = 52.0 + 48.0 * (L.nt - 1) + 48.0 * L.nt +
                           (L.lagrange ? 0.0 : 8.0 * (2 * L.nt + 1));
  Prof P(c, REG_KC_MATVEC, (double)L.g.N * per_point);
  check(c, launch_gn_matvec(a, c->st), "persistent matvec launch");
}

// the GN data term b~ in one launch (flow.cu)
void data_term_flow(reg_ctx* c, Level& L, const float* vt, float* b) {
  LevelScope ls(c, L);
  FlowArgs a{};
  a.n1 = L.g.n1;
  a.n2 = L.g.n2;
  a.log1 = L.g.log1;
  a.nt = L.nt;
  a.N = L.g.N;
  a.ht = L.ht;
  a.tiles_x = L.flow_tx;
  a.tiles_y = L.flow_ty;
  a.vt = vt;
  a.dX = L.dX;
  a.dY = L.dY;
  a.delta = L.delta;
  a.delta_bar = L.delta_bar;
  a.gm = L.gm;
  a.G = L.G;
  a.buf0 = L.fA;
  a.buf1 = L.fB;
  a.b = b;
  a.flags = L.flow_flags;
  a.err = c->barerr;
  a.dmax = L.flow_dmax;
  a.inject = c->opt.inject_barrier_timeout ? 1 : 0;
  // algorithmic bytes per point (each field read or written once): per
  // incremental state step G_j, grad m_j, m~ in and out (24), per adjoint
  // step grad m_j, lambda~ in and out (16), once: dX, dY, v~, div v,
  // div v(Y_D), b~ (40) and v~(X_D) kept on chip, minus the reads and writes
  // the ends of the chain do not make (m~_0 and lambda~_0: 8)
  const double per_point = 24.0 * L.nt + 16.0 * L.nt + 40.0 - 8.0;
  Prof P(c, REG_KC_MATVEC, (double)L.g.N * per_point);
  check(c, launch_gn_flow(a, c->st), "flow matvec launch");
}

// the launch sequence of one GN matvec; needs ensure_G(c, L) beforehand
void hessian_full(reg_ctx* c, Level& L, const float* vt, float* out);

void hessian_core(reg_ctx* c, Level& L, const float* vt, float* out, bool data_only) {
  LevelScope ls(c, L);
  if (c->full_newton && !data_only && &L == &c->fine) {
    hessian_full(c, L, vt, out);
    return;
  }
  if (c->persistent) {
    const size_t N2 = 2 * (size_t)L.g.N;
    if (data_only) {
      data_term_persistent(c, L, vt, out);
    } else {
      data_term_persistent(c, L, vt, L.b);
      if (has_K(c))
        finish_hessian_K(c, L, vt, out);
      else
        spectral(c, L, SPOP_REGPOW, 1.0, vt, 1, 2, out, 1, L.b);
    }
    (void)N2;
    return;
  }
  // beta A v~: its forward transforms depend only on v~ and run on the side
  // stream while the transport steps (which use no FFT workspace) run here
  const bool fork = !data_only && !has_K(c);
  if (L.flow) {
    if (fork) on_side(c, [&] { spectral_fwd(c, L, SPOP_REGPOW, 1.0, vt, 1, 2, 1); });
    data_term_flow(c, L, vt, data_only ? out : L.b);
    if (data_only) return;
    if (has_K(c)) {
      finish_hessian_K(c, L, vt, out);
    } else {
      join_side(c);
      spectral_inv(c, L, 1, 2, out, 1, L.b);
    }
    return;
  }
  const GridDims& gd = L.g;
  const size_t N = (size_t)gd.N;
  const int nt = L.nt;
  const float ht = L.ht;
  const int lg = L.lagrange;
  if (fork) on_side(c, [&] { spectral_fwd(c, L, SPOP_REGPOW, 1.0, vt, 1, 2, 1); });
  // the time integral b~ accumulates in the output itself when only the data
  // term is wanted (out must not alias vt)
  float* bacc = data_only ? out : L.b;
  float* mt = L.fA;
  float* mt2 = L.fB;
  float* lt = nullptr;
  float* lt2 = nullptr;
  if (L.fuse_w) {
    // prefilter of v~, v~(X_D) and m~_1 in one kernel; later steps prefilter
    // m~_{j-1} inside the step; the last one also writes lambda~_nt and
    // starts b~ (the work of k_adjoint_init)
    {
      Prof P(c, REG_KC_INCSTATE_STEP, kIncStepBytes(1, nt) * N);
      launch_incstate_first_fused(L.fuse_w, gd.n1, gd.n2, ht, vt, L.dX, L.G, L.gm + 2 * N, L.vtD,
                                  mt2, c->st);
    }
    std::swap(mt, mt2);
    for (int j = 2; j <= nt; ++j) {
      const bool last = (j == nt);
      Prof P(c, REG_KC_INCSTATE_STEP, kIncStepBytes(j, nt) * N);
      incstate_fused(c, L, mt, vt, L.G + 2 * (j - 1) * N, L.gm + 2 * j * N, mt2,
                     last ? bacc : nullptr);
      std::swap(mt, mt2);
    }
    if (nt >= 2) {   // mt holds lambda~_nt
      lt = mt;
      lt2 = mt2;
    }
  } else {
    // v~(X_D) is gathered by the first step; the last one (nt >= 2) also
    // writes lambda~_nt and starts b~
    const float* cvt = coefficients(c, L, vt, 2, L.c2);
    for (int j = 1; j <= nt; ++j) {
      const float* cm = (j == 1) ? nullptr : coefficients(c, L, mt, 1, L.coef);
      const bool last = (j == nt && nt >= 2);
      {
        Prof P(c, REG_KC_INCSTATE_STEP, kIncStepBytes(j, nt) * N);
        launch_incstate_step(L.tile_inc, gd.n1, gd.n2, ht, cm, L.dX, vt, L.vtD, L.G + 2 * (j - 1) * N,
                             L.gm + 2 * j * N, mt2, j == 1, lg, c->st, j == 1 ? cvt : nullptr,
                             last ? L.gm + 2 * nt * N : nullptr, last ? bacc : nullptr);
      }
      std::swap(mt, mt2);
    }
    if (nt >= 2) {   // mt holds lambda~_nt
      lt = mt;
      lt2 = mt2;
    }
  }
  check_launch(c, "incremental state");
  if (!lt) {
    // lambda~_nt = -m~_nt
    lt = mt2;
    {
      Prof P(c, REG_KC_VECTOR, 24.0 * N);
      launch_adjoint_init(gd.n1, gd.n2, 0.5f * ht, nullptr, mt, L.gm + 2 * nt * N, lt, bacc, 1.f, c->st);
    }
    lt2 = mt;
  }
  for (int j = nt - 1; j >= 0; --j) {
    const float wb = ht * (j == 0 ? 0.5f : 1.0f);
    if (L.fuse_w) {   // prefilter of lambda~_{j+1} inside the step kernel
      Prof P(c, REG_KC_ADJOINT_STEP, kAdjStepBytes(j == nt - 1) * N);
      adjoint_fused(c, L, wb, lt, L.gm + 2 * j * N, lt2, bacc);
      std::swap(lt, lt2);
      continue;
    }
    const float* cl = coefficients(c, L, lt, 1, L.coef);
    {
      Prof P(c, REG_KC_ADJOINT_STEP, kAdjStepBytes(j == nt - 1) * N);
      launch_adjoint_step(L.tile_adj, gd.n1, gd.n2, ht, wb, cl, L.dY, L.delta, L.delta_bar,
                          L.gm + 2 * j * N, lt2, bacc, lg, c->st);
    }
    std::swap(lt, lt2);
  }
  check_launch(c, "incremental adjoint");
  if (data_only) {
    // b~ is already in out
  } else if (has_K(c)) {
    finish_hessian_K(c, L, vt, out);
  } else {
    join_side(c);
    spectral_inv(c, L, 1, 2, out, 1, L.b);
  }
}

void set_images_level(reg_ctx* c, Level& L) {
  spectral(c, L, SPOP_GRAD, 0.0, L.mT, 1, 1, L.gm, 2, nullptr);
  L.have_images = true;
  L.have_v = L.have_gm = L.have_div = L.have_G = false;
}

// ---------------------------------------------------------------------------
// preconditioners and Krylov solvers

// Full-Newton Hessian matvec (eq. hessian-matvec with its lambda terms):
// H v~ = beta A v~ + K[int_0^1 lambda~ grad m + lambda grad m~ dt], lambda~
// from eq. inc-adj-slm with the div(lambda v~) source. Uses the adjoint
// history of the gradient at the cached velocity (recomputed if missing),
// keeps m~_j, and runs the steps unfused (the source is a second gathered
// field). Problem grid only.
void hessian_full(reg_ctx* c, Level& L, const float* vt, float* out) {
  const GridDims& gd = L.g;
  const size_t N = (size_t)gd.N;
  const int nt = L.nt;
  const float ht = L.ht;
  const int lg = L.lagrange;
  ensure_G(c, L);
  if (!L.have_lam) {
    objective(c, L);
    gradient(c, L, L.w2);
  }
  // incremental state, m~_j kept in mt_hist (m~_0 = 0 is never read)
  if (L.fuse_w) {
    {
      Prof P(c, REG_KC_INCSTATE_STEP, 44.0 * N);
      launch_incstate_first_fused(L.fuse_w, gd.n1, gd.n2, ht, vt, L.dX, L.G, L.gm + 2 * N, L.vtD,
                                  L.mt_hist + N, c->st);
    }
    for (int j = 2; j <= nt; ++j) {
      Prof P(c, REG_KC_INCSTATE_STEP, 48.0 * N);
      launch_incstate_fused(L.fuse_w, gd.n1, gd.n2, ht, L.mt_hist + (j - 1) * N, L.dX, vt, L.vtD,
                            L.G + 2 * (j - 1) * N, L.gm + 2 * j * N, L.mt_hist + j * N, nullptr,
                            nullptr, c->st);
    }
  } else {
    const float* cvt = coefficients(c, L, vt, 2, L.c2);
    for (int j = 1; j <= nt; ++j) {
      const float* cm = (j == 1) ? nullptr : coefficients(c, L, L.mt_hist + (j - 1) * N, 1, L.coef);
      Prof P(c, REG_KC_INCSTATE_STEP, (j == 1 ? 52.0 : 48.0) * N);
      launch_incstate_step(L.tile_inc, gd.n1, gd.n2, ht, cm, L.dX, vt, L.vtD, L.G + 2 * (j - 1) * N,
                           L.gm + 2 * j * N, L.mt_hist + j * N, j == 1, lg, c->st,
                           j == 1 ? cvt : nullptr, nullptr, nullptr);
    }
  }
  check_launch(c, "incremental state");
  // s_j = div(lambda_j v~), j = 0..nt, and grad m~_j, j = 1..nt
  {
    Prof P(c, REG_KC_VECTOR, 16.0 * (nt + 1) * N);
    launch_lam_times_vt((long long)N, nt + 1, L.lam_hist, vt, L.prod, c->st);
  }
  spectral(c, L, SPOP_DIV, 0.0, L.prod, 2, nt + 1, L.src, 1, nullptr);
  spectral(c, L, SPOP_GRAD, 0.0, L.mt_hist + N, 1, nt, L.gmt, 2, nullptr);
  // lambda~_nt = -m~_nt and the first term of the time integral
  float* lt = L.fA;
  float* lt2 = L.fB;
  {
    Prof P(c, REG_KC_VECTOR, 36.0 * N);
    launch_fn_adjoint_init((long long)N, 0.5f * ht, L.mt_hist + nt * N, L.gm + 2 * nt * N,
                           L.lam_hist + nt * N, L.gmt + 2 * (nt - 1) * N, lt, L.b, c->st);
  }
  for (int j = nt - 1; j >= 0; --j) {
    const float wb = ht * (j == 0 ? 0.5f : 1.0f);
    const float* cl = coefficients(c, L, lt, 1, L.coef);
    const float* cs = coefficients(c, L, L.src + (j + 1) * N, 1, L.c2);
    {
      Prof P(c, REG_KC_ADJOINT_STEP, 68.0 * N);
      launch_fn_adjoint_step(gd.n1, gd.n2, ht, wb, cl, cs, L.dY, L.delta, L.delta_bar,
                             L.src + j * N, L.gm + 2 * j * N, L.lam_hist + j * N,
                             j ? L.gmt + 2 * (j - 1) * N : nullptr, lt2, L.b, lg, c->st);
    }
    std::swap(lt, lt2);
  }
  check_launch(c, "incremental adjoint (full Newton)");
  if (has_K(c))
    finish_hessian_K(c, L, vt, out);
  else
    spectral(c, L, SPOP_REGPOW, 1.0, vt, 1, 2, out, 1, L.b);
}

// (I + (beta A_c)^-1/2 Q_c (beta A_c)^-1/2) s on the coarse level.
void coarse_split_op(reg_ctx* c, const float* s, float* out) {
  LevelScope ls(c, c->coarse);
  Level& C = c->coarse;
  spectral(c, C, SPOP_REGPOW, -0.5, s, 1, 2, c->cu, 1, nullptr);
  hessian_core(c, C, c->cu, c->cq, true);
  if (has_K(c))
    spectral(c, C, regpow_K_op(c), -0.5, c->cq, 2, 1, out, 2, s);
  else
    spectral(c, C, SPOP_REGPOW, -0.5, c->cq, 1, 2, out, 1, s);
  ++c->coarse_matvecs;
}

// Largest eigenvalue of a symmetric tridiagonal matrix by Sturm bisection.
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
      d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::fmax(1.0, std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= m) hi = mid; else lo = mid;
  }
  return hi;
}

void estimate_eigenvalues(reg_ctx* c) {
  Level& C = c->coarse;
  const long long n = 2 * C.g.N;
  // coarse problem at v = 0
  launch_fill(C.w1, n, 0.f, c->st);
  set_velocity(c, C, C.w1);
  ensure_G(c, C);
  float* q = c->cp;
  float* qprev = c->cz;
  float* w = c->cd;
  launch_splitmix(q, n, c->opt.lanczos_seed, c->st);
  if (c->incompressible) {   // start (and stay) among divergence-free fields
    spectral(c, C, SPOP_LERAY, 0.0, q, 2, 1, C.w2, 2, nullptr);
    check(c, cudaMemcpyAsync(q, C.w2, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  }
  const double nq = std::sqrt(dot_sync(c, q, q, n, S_A));
  launch_lincomb(n, (float)(1.0 / nq), q, 0.f, nullptr, q, c->st);
  launch_fill(qprev, n, 0.f, c->st);
  std::vector<double> al, be;
  double beta = 0.0;
  for (int k = 0; k < c->opt.lanczos_steps; ++k) {
    coarse_split_op(c, q, w);
    const double alpha = dot_sync(c, q, w, n, S_A);
    launch_lincomb(n, 1.f, w, (float)-alpha, q, w, c->st);
    launch_lincomb(n, 1.f, w, (float)-beta, qprev, w, c->st);
    al.push_back(alpha);
    const double bn = std::sqrt(dot_sync(c, w, w, n, S_B));
    if (!(bn > 1e-12 * std::fabs(alpha))) break;
    be.push_back(bn);
    std::swap(qprev, q);                       // qprev <- q
    launch_lincomb(n, (float)(1.0 / bn), w, 0.f, nullptr, q, c->st);  // q <- w / beta
    beta = bn;
  }
  be.resize(al.size() > 0 ? al.size() - 1 : 0);
  const double rmax = tridiag_max_eig(al, be);
  const int p = c->opt.reg_norm;
  const double kn = 0.25 * ((double)C.g.n1 * C.g.n1 + (double)C.g.n2 * C.g.n2);
  const double gmax = std::pow(kn, p);
  c->emin = 1.0 + 1.0 / (c->beta * gmax);
  c->emax = rmax * c->opt.emax_safety;
  c->eig_beta = c->beta;
  c->have_eig = true;
}

// (I + (beta A_c)^-1 Q_c) u on the coarse level: the split operator above
// conjugated by (beta A_c)^1/2, same spectrum, one spectral operation less.
void coarse_op_u(reg_ctx* c, const float* u, float* out, const ChebEpilogue* cheb = nullptr) {
  LevelScope ls(c, c->coarse);
  Level& C = c->coarse;
  hessian_core(c, C, u, c->cq, true);
  if (has_K(c))
    spectral(c, C, regpow_K_op(c), -1.0, c->cq, 2, 1, out, 2, u, cheb);
  else
    spectral(c, C, SPOP_REGPOW, -1.0, c->cq, 1, 2, out, 1, u, cheb);
  ++c->coarse_matvecs;
}

void cheb(reg_ctx* c, const float* rhs, float* x) {
  LevelScope ls(c, c->coarse);
  const long long n = 2 * c->coarse.g.N;
  const double theta = 0.5 * (c->emax + c->emin), delta = 0.5 * (c->emax - c->emin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  check(c, cudaMemcpyAsync(c->cr, rhs, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  launch_lincomb(n, (float)(1.0 / theta), rhs, 0.f, nullptr, c->cd, c->st);
  check(c, cudaMemcpyAsync(x, c->cd, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  for (int it = 1; it < c->opt.cheb_iters; ++it) {
    // the operator application ends in the iteration's vector work
    // (r -= A d; d = a d + b r; x += d) inside its last FFT pass
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    ChebEpilogue ce;
    ce.r = c->cr;
    ce.d = c->cd;
    ce.x = x;
    ce.a = (float)(rho_new * rho);
    ce.b = (float)(2.0 * rho_new / delta);
    coarse_op_u(c, c->cd, c->cAd, &ce);
    rho = rho_new;
  }
  check_launch(c, "chebyshev");
}

struct PcgResult {
  int iters = 0, matvecs = 0;
  bool negcurv = false;
  double relres = 1.0;
};

// PCG (Hestenes-Stiefel), zero initial guess, on vectors of length n.
template <typename Op, typename Prec>
PcgResult pcg(reg_ctx* c, long long n, Op A, Prec M, const float* rhs, float* x, float* r,
              float* z, float* p, float* q, double rtol, int maxit, int sb) {
  PcgResult res;
  const int S_RZ = sb + P_RZ, S_RZNEW = sb + P_RZNEW, S_PQ = sb + P_PQ, S_RR = sb + P_RR,
            S_BB = sb + P_BB;
  launch_fill(x, n, 0.f, c->st);
  check(c, cudaMemcpyAsync(r, rhs, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  const double bnorm = std::sqrt(dot_sync(c, rhs, rhs, n, S_BB));
  if (!(bnorm > 0.0)) {
    res.relres = 0.0;
    return res;
  }
  M(r, z);
  check(c, cudaMemcpyAsync(p, z, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  dot_async(c, r, z, n, S_RZ);
  for (int it = 0; it < maxit; ++it) {
    A(p, q);
    ++res.matvecs;
    // p.q, the update (skipped on the device when p.q <= 0) and r.r are
    // queued together and read back with one synchronisation
    dot_async(c, p, q, n, S_PQ);
    {
      Prof P(c, REG_KC_VECTOR, 24.0 * n);
      launch_pcg_update(n, slot(c, S_RZ), slot(c, S_PQ), p, q, x, r, c->st);
    }
    dot_async(c, r, r, n, S_RR);
    read_slots(c, S_PQ, 2);
    const double pq = c->hsc[S_PQ], rr = c->hsc[S_RR];
    if (!(pq > 0.0)) {   // negative curvature: x and r were left unchanged
      res.negcurv = true;
      if (it == 0) check(c, cudaMemcpyAsync(x, z, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
      break;
    }
    res.iters = it + 1;
    res.relres = std::sqrt(rr) / bnorm;
    if (res.relres <= rtol) break;
    M(r, z);
    dot_async(c, r, z, n, S_RZNEW);
    {
      Prof P(c, REG_KC_VECTOR, 12.0 * n);
      launch_pcg_direction(n, slot(c, S_RZNEW), slot(c, S_RZ), z, p, c->st);
    }
    check(c, cudaMemcpyAsync(slot(c, S_RZ), slot(c, S_RZNEW), sizeof(double), cudaMemcpyDeviceToDevice, c->st), "copy");
    check_launch(c, "pcg");
  }
  return res;
}


void coarse_velocity(reg_ctx* c) {
  resample(c, c->fine, c->coarse, SPOP_SCALE, 0.0, c->fine.v, 2, c->coarse.w2, nullptr);
  set_velocity(c, c->coarse, c->coarse.w2);
}

void precond(reg_ctx* c, const float* r, float* z) {
  Level& F = c->fine;
  const long long n = 2 * F.g.N;
  if (!c->two_level) {
    spectral(c, F, SPOP_REGPOW, -1.0, r, 1, 2, z, 1, nullptr);
    return;
  }
  Level& C = c->coarse;
  const long long nc = 2 * C.g.N;
  if (c->opt.pc_solver == REG_PCSOLVER_CHEB) {
    // CHEB(k) is a polynomial in the operator, so it can run on
    // (beta A_c)^-1/2 (split operator) (beta A_c)^1/2 = I + (beta A_c)^-1 Q_c
    // with u = (beta A_c)^-1/2 s: right-hand side R (beta A)^-1 r, and the
    // result enters the prolongation without a further (beta A)^-1/2.
    resample(c, F, C, SPOP_REGPOW, -1.0, r, 2, c->crhs, nullptr);
    // high band (beta A)^-1/2 H (beta A)^-1/2 r = (beta A)^-1 H r -> F.w1 on
    // the side stream, concurrently with the coarse solve (it uses only the
    // fine grid's FFT workspace, the coarse solve only the coarse grid's)
    on_side(c, [&] { spectral(c, F, SPOP_REGPOW_HIGH, -1.0, r, 1, 2, F.w1, 1, nullptr); });
    cheb(c, c->crhs, c->cx);
    join_side(c);
    resample(c, C, F, SPOP_SCALE, 0.0, c->cx, 2, z, F.w1);
    return;
  }
  // high band: (beta A)^-1/2 H (beta A)^-1/2 r = (beta A)^-1 H r -> F.w1
  spectral(c, F, SPOP_REGPOW_HIGH, -1.0, r, 1, 2, F.w1, 1, nullptr);
  // r' = (beta A)^-1/2 r; restricted low band -> crhs
  resample(c, F, C, SPOP_REGPOW, -0.5, r, 2, c->crhs, nullptr);
  {
    LevelScope ls(c, C);
    auto A = [&](const float* s, float* o) { coarse_split_op(c, s, o); };
    auto I = [&](const float* s, float* o) {
      check(c, cudaMemcpyAsync(o, s, nc * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
    };
    pcg(c, nc, A, I, c->crhs, c->cx, c->cr, c->cz, c->cp, c->cq, c->opt.pc_eps * c->eta,
        c->opt.max_pcg, S_PCG_INNER);
  }
  // z = (beta A)^-1/2 P s_c + (beta A)^-1 H r
  resample(c, C, F, SPOP_REGPOW, -0.5, c->cx, 2, z, F.w1);
  (void)n;
}

PcgResult kkt(reg_ctx* c, const float* rhs, double rtol, int maxit, float* x) {
  Level& F = c->fine;
  const long long n = 2 * F.g.N;
  if (c->two_level) {
    if (!c->have_eig) {
      estimate_eigenvalues(c);
    } else if (c->eig_beta != c->beta) {
      const double s = c->eig_beta / c->beta;
      c->emin = 1.0 + (c->emin - 1.0) * s;
      c->emax = 1.0 + (c->emax - 1.0) * s;
      c->eig_beta = c->beta;
    }
    coarse_velocity(c);
    ensure_G(c, c->coarse);
  }
  ensure_G(c, F);
  // the full-Newton matvec reads the adjoint history of this velocity; a
  // replayed graph cannot recompute it, so it is brought up to date here
  if (c->full_newton && !F.have_lam) {
    objective(c, F);
    gradient(c, F, F.w2);
  }
  auto A = [&](const float* p, float* q) {
    graphed(c, graph_key(c, "mv", p, q), [&] { hessian_core(c, F, p, q, false); });
  };
  auto M = [&](const float* r, float* z) {
    if (c->two_level && c->opt.pc_solver == REG_PCSOLVER_CHEB) {
      if (!graphed(c, graph_key(c, "pc", r, z), [&] { precond(c, r, z); }))
        c->coarse_matvecs += c->opt.cheb_iters - 1;   // replayed: count its coarse matvecs
    } else
      precond(c, r, z);
  };
  return pcg(c, n, A, M, rhs, x, c->kr, c->kz, c->kp, c->kq, rtol, maxit, S_PCG_OUTER);
}

double max_abs_sync(reg_ctx* c, const float* a, long long n, int s) {
  {
    Prof P(c, REG_KC_REDUCE, 4.0 * n);
    launch_maxabs(a, n, c->partialf, slot(c, s), c->st);
  }
  check_launch(c, "maxabs");
  read_slots(c, s, 1);
  return c->hsc[s];
}

void require_images(reg_ctx* c) {
  if (!c->fine.have_images) fail(c, REG_ESTATE, "reg_set_images has not been called");
}

// full objective + gradient at v on the fine level
double objective_gradient(reg_ctx* c, const float* v, float* g) {
  set_velocity(c, c->fine, v);
  const double J = objective(c, c->fine);
  if (g) gradient(c, c->fine, g);
  return J;
}

void ensure_gref(reg_ctx* c) {
  if (c->have_gref) return;
  Level& F = c->fine;
  const long long n = 2 * F.g.N;
  launch_fill(c->vtrial, n, 0.f, c->st);
  c->J_zero = objective_gradient(c, c->vtrial, c->gcur);
  c->gref_inf = max_abs_sync(c, c->gcur, n, S_GINF);
  c->gref_2 = std::sqrt(dot_sync(c, c->gcur, c->gcur, n, S_G2));
  c->have_gref = true;
}

// Device buffers are read and written with 8- and 16-byte vector accesses;
// one that starts off a 16-byte boundary is rejected on the host.
bool unaligned(std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (reinterpret_cast<uintptr_t>(p) & 15u) return true;
  return false;
}

reg_status reject_unaligned(reg_ctx* c) {
  c->err = "device buffers must start on a 16-byte boundary";
  return REG_EINVAL;
}


reg_status guarded(reg_ctx* c, const std::function<void()>& body) {
  if (!c) return REG_EINVAL;
  LaunchModeScope mode(c->opt.programmatic_launch ? 1 : 0);
  ReducePrecisionScope prec(c->opt.precision == REG_PRECISION_FP32 ? 1 : 0);
  try {
    body();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      c->err = std::string("CUDA: ") + cudaGetErrorString(e);
      return REG_ECUDA;
    }
    return REG_OK;
  } catch (const CudaError& e) {
    return e.s;
  }
}
}  // namespace

// ===========================================================================
// C ABI

extern "C" {

reg_status reg_default_options(reg_options* o) {
  if (!o) return REG_EINVAL;
  o->reg_norm = REG_H1;
  o->interp = REG_INTERP_SPLINE;
  o->precond = REG_PC_2L;
  o->pc_solver = REG_PCSOLVER_CHEB;
  o->cheb_iters = 10;
  o->pc_eps = 0.1;
  o->gabs = 1e-5;
  o->max_newton = 50;
  o->max_pcg = 100;
  o->lanczos_steps = 30;
  o->emax_safety = 1.05;
  o->lanczos_seed = 20160407ULL;
  o->max_backtracks = 10;
  o->armijo_c1 = 1e-4;
  o->persistent_matvec = 0;
  o->inject_barrier_timeout = 0;
  o->programmatic_launch = 1;
  o->fused_transport = 1;
  o->coarse_nt = 0;
  o->coarse_interp = -1;
  o->step_tile = -1;
  o->incompressible = 0;
  o->hessian = 0;
  o->precision = REG_PRECISION_FP64;
  o->use_graphs = 1;
  o->flow_matvec = 0;
  o->beta_w = 0.0;
  o->graph_pdl = 0;
  return REG_OK;
}

// grid sizes: 2^k in [32, 2048] or 3 * 2^k in [96, 1536] (the FFT's line
// lengths; multiples of 32 for the prefilter tiles)
static bool size_ok(int n) { return n % 32 == 0 && fft_size_supported(n); }

reg_status reg_create(reg_grid grid, int nt, double beta, const reg_options* opt, reg_ctx** out) {
  if (!out) return REG_EINVAL;
  *out = nullptr;
  if (!size_ok(grid.n1) || !size_ok(grid.n2) || nt < 1 || nt > 4096 || !(beta > 0.0))
    return REG_EINVAL;
  reg_options o;
  if (opt) o = *opt; else reg_default_options(&o);
  if (o.reg_norm < 1 || o.reg_norm > 3 || (o.interp != 0 && o.interp != 1) ||
      (o.precond != 0 && o.precond != 1) || (o.pc_solver != 0 && o.pc_solver != 1) ||
      o.cheb_iters < 1 || o.max_pcg < 1 || o.lanczos_steps < 1 || o.max_newton < 0 ||
      o.coarse_nt < 0 || o.coarse_nt > 4096 || o.coarse_interp < -1 || o.coarse_interp > 1 ||
      o.step_tile < -1 || o.step_tile > kStepTiles ||
      (o.incompressible != 0 && o.incompressible != 1) || (o.hessian != 0 && o.hessian != 1) ||
      (o.hessian == 1 && o.persistent_matvec != 0) ||
      (o.precision != REG_PRECISION_FP64 && o.precision != REG_PRECISION_FP32) ||
      (o.use_graphs != 0 && o.use_graphs != 1) || (o.flow_matvec != 0 && o.flow_matvec != 1) ||
      !(o.beta_w >= 0.0 && o.beta_w < 1e30) || (o.beta_w > 0.0 && o.incompressible) ||
      o.graph_pdl < 0 || o.graph_pdl > 2)
    return REG_EINVAL;
  if (o.precond == REG_PC_2L && (!size_ok(grid.n1 / 2) || !size_ok(grid.n2 / 2) ||
                                 grid.n1 % 2 || grid.n2 % 2))
    return REG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return REG_ECUDA;
  reg_ctx* c = new reg_ctx();
  c->device = dev;
  c->opt = o;
  c->beta = beta;
  c->nt = nt;
  c->two_level = (o.precond == REG_PC_2L);
  c->incompressible = (o.incompressible != 0);
  c->full_newton = (o.hessian == REG_HESSIAN_FULL);
  c->beta_w = o.beta_w;
  c->graphs = (o.use_graphs != 0);
  c->fine.lagrange = (o.interp == REG_INTERP_LAGRANGE);
  c->coarse.lagrange = o.coarse_interp < 0 ? c->fine.lagrange : (o.coarse_interp == REG_INTERP_LAGRANGE);
  c->persistent = (o.persistent_matvec != 0);
  const reg_status s = guarded(c, [&] {
    fused_init();   // shared-memory limit of the fused step kernels on this device
    alloc_level(c, c->fine, grid.n1, grid.n2, nt);
    if (c->two_level)
      alloc_level(c, c->coarse, grid.n1 / 2, grid.n2 / 2, o.coarse_nt > 0 ? o.coarse_nt : nt);
    if (c->full_newton) {
      Level& F = c->fine;
      const size_t N = (size_t)F.g.N, L1 = (size_t)nt + 1;
      F.lam_hist = dalloc<float>(c, L1 * N);
      F.mt_hist = dalloc<float>(c, L1 * N);
      F.src = dalloc<float>(c, L1 * N);
      F.gmt = dalloc<float>(c, 2 * (size_t)nt * N);
      F.prod = dalloc<float>(c, 2 * L1 * N);
    }
    choose_step_tiles(c, c->fine);
    if (c->two_level) choose_step_tiles(c, c->coarse);
    check(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "capture stream");
    check(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "side stream");
    check(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "event");
    check(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "event");
    c->dsc = dalloc<double>(c, kScalars);
    void* h = nullptr;
    check(c, cudaMallocHost(&h, kScalars * sizeof(double)), "cudaMallocHost");
    c->hsc = static_cast<double*>(h);
    void* hf = nullptr;
    check(c, cudaMallocHost(&hf, sizeof(int)), "cudaMallocHost");
    c->hflag = static_cast<int*>(hf);
    c->partial = dalloc<double>(c, reduce_partials());
    c->partialf = dalloc<float>(c, reduce_partials());
    c->dflag = dalloc<int>(c, 1);
    c->bar = dalloc<unsigned>(c, 2);
    c->barerr = dalloc<int>(c, 1);
    check(c, cudaMemset(c->bar, 0, 2 * sizeof(unsigned)), "memset");
    check(c, cudaMemset(c->barerr, 0, sizeof(int)), "memset");
    void* he = nullptr;
    check(c, cudaMallocHost(&he, sizeof(int)), "cudaMallocHost");
    c->hbarerr = static_cast<int*>(he);
    *c->hbarerr = 0;
    const size_t n = 2 * (size_t)c->fine.g.N;
    c->kx = dalloc<float>(c, n);
    c->kr = dalloc<float>(c, n);
    c->kz = dalloc<float>(c, n);
    c->kp = dalloc<float>(c, n);
    c->kq = dalloc<float>(c, n);
    c->vtrial = dalloc<float>(c, n);
    c->gcur = dalloc<float>(c, n);
    c->vt_tmp = dalloc<float>(c, n);
    if (c->two_level) {
      const size_t nc = 2 * (size_t)c->coarse.g.N;
      c->cx = dalloc<float>(c, nc);
      c->cr = dalloc<float>(c, nc);
      c->cd = dalloc<float>(c, nc);
      c->cAd = dalloc<float>(c, nc);
      c->crhs = dalloc<float>(c, nc);
      c->cu = dalloc<float>(c, nc);
      c->cq = dalloc<float>(c, nc);
      c->cz = dalloc<float>(c, nc);
      c->cp = dalloc<float>(c, nc);
    }
    check(c, cudaDeviceSynchronize(), "create");
  });
  if (s != REG_OK) {
    reg_destroy(c);
    return s;
  }
  *out = c;
  return REG_OK;
}

reg_status reg_destroy(reg_ctx* c) {
  if (!c) return REG_OK;
  if (c->st) cudaStreamSynchronize(c->st);
  drop_graphs(c);   // returns the graphs' profiling events to the pool
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (void* p : c->allocs) cudaFree(p);
  if (c->hsc) cudaFreeHost(c->hsc);
  if (c->hflag) cudaFreeHost(c->hflag);
  if (c->hbarerr) cudaFreeHost(c->hbarerr);
  delete c;
  return REG_OK;
}

reg_status reg_set_stream(reg_ctx* c, void* stream) {
  if (!c) return REG_EINVAL;
  c->st = static_cast<cudaStream_t>(stream);
  return REG_OK;
}

const char* reg_last_error(const reg_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

reg_status reg_set_images(reg_ctx* c, const float* mR, const float* mT) {
  if (!c || !mR || !mT) return REG_EINVAL;
  if (unaligned({mR, mT})) return reject_unaligned(c);
  return guarded(c, [&] {
    Level& F = c->fine;
    const size_t N = (size_t)F.g.N;
    check(c, cudaMemcpyAsync(F.mR, mR, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy m_R");
    check(c, cudaMemcpyAsync(F.mT, mT, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy m_T");
    set_images_level(c, F);
    if (c->two_level) {
      Level& C = c->coarse;
      resample(c, F, C, SPOP_SCALE, 0.0, F.mR, 1, C.mR, nullptr);
      resample(c, F, C, SPOP_SCALE, 0.0, F.mT, 1, C.mT, nullptr);
      set_images_level(c, C);
    }
    c->have_eig = false;
    c->have_gref = false;
  });
}

reg_status reg_set_beta(reg_ctx* c, double beta) {
  if (!c || !(beta > 0.0)) return REG_EINVAL;
  c->beta = beta;  // eigenvalue bounds are rescaled lazily in kkt()
  return REG_OK;
}

reg_status reg_transport(reg_ctx* c, const float* v, const float* m0, float* m1) {
  if (!c || !v || !m0 || !m1) return REG_EINVAL;
  if (unaligned({v, m0, m1})) return reject_unaligned(c);
  return guarded(c, [&] {
    Level& F = c->fine;
    const size_t N = (size_t)F.g.N;
    // the state solve uses m_T as initial condition: run it on a copy
    F.have_v = F.have_gm = F.have_div = F.have_G = false;
    check(c, cudaMemcpyAsync(F.w2, F.mT, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "save m_T");
    check(c, cudaMemcpyAsync(F.mT, m0, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy m0");
    set_velocity(c, F, v);
    check(c, cudaMemcpyAsync(m1, F.m + F.nt * N, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy m1");
    check(c, cudaMemcpyAsync(F.mT, F.w2, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "restore m_T");
    F.have_v = F.have_gm = F.have_div = F.have_G = false;
  });
}

// RK2A comparator (Appendix "RK2A derivation"): nt Heun steps of the
// antisymmetric-form state equation (sign -1) or of its adjoint backward in
// time (sign +1), pseudospectral derivatives on the problem grid.
static void rk2a_solve(reg_ctx* c, const float* v, const float* u0, float* u1, int nt, float sign) {
  Level& F = c->fine;
  const size_t N = (size_t)F.g.N;
  if (!c->rk2a) c->rk2a = dalloc<float>(c, 9 * N);
  float* delta = c->rk2a;
  float* m = delta + N;
  float* ms = m + N;
  float* k1 = ms + N;
  float* g = k1 + N;
  float* prod = g + 2 * N;
  float* dv = prod + 2 * N;
  spectral(c, F, SPOP_DIV, 0.0, v, 2, 1, delta, 1, nullptr);
  check(c, cudaMemcpyAsync(m, u0, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  const float ht = 1.0f / (float)nt;
  auto stage = [&](const float* u, float a, const float* kprev, float b, float* out, float* kout) {
    launch_lam_times_vt((long long)N, 1, u, v, prod, c->st);   // u v
    spectral(c, F, SPOP_GRAD, 0.0, u, 1, 1, g, 2, nullptr);
    spectral(c, F, SPOP_DIV, 0.0, prod, 2, 1, dv, 1, nullptr);
    launch_rk2a_stage((long long)N, sign, u, g, v, dv, delta, m, a, kprev, b, out, kout, c->st);
  };
  for (int j = 0; j < nt; ++j) {
    stage(m, ht, nullptr, 0.f, ms, k1);            // u* = u + h_t k1
    stage(ms, 0.5f * ht, k1, 0.5f * ht, m, nullptr);   // u <- u + h_t/2 (k1 + k2)
  }
  check_launch(c, "RK2A solve");
  check(c, cudaMemcpyAsync(u1, m, N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
}

// Deformation map (§2: m_1 = m_T o y): u = y - x as the composition of the
// nt departure maps X_D of v, u_j = u_{j-1}(X_D) + (X_D - x) from u_0 = 0,
// and optionally det grad y (spectral derivatives of u).
static void deformation_map(reg_ctx* c, const float* v, float* u, float* det) {
  Level& F = c->fine;
  const GridDims& g = F.g;
  const size_t N = (size_t)g.N;
  if (!c->defmap) c->defmap = dalloc<float>(c, 10 * N);
  float* dX = c->defmap;
  float* ua = dX + 2 * N;
  float* ub = ua + 2 * N;
  float* gr = ub + 2 * N;
  const float h1 = (float)F.h1, h2 = (float)F.h2;
  const float* cv = coefficients(c, F, v, 2, F.c2);
  launch_departure(g.n1, g.n2, F.ht, v, cv, dX, nullptr, F.lagrange, c->st);
  launch_lincomb((long long)N, h1, dX, 0.f, nullptr, ua, c->st);
  launch_lincomb((long long)N, h2, dX + N, 0.f, nullptr, ua + N, c->st);
  for (int j = 2; j <= F.nt; ++j) {
    const float* cu = coefficients(c, F, ua, 2, F.c2);
    launch_gather(g.n1, g.n2, cu, dX, ub, 2, (long long)N, F.lagrange, c->st);
    launch_lincomb((long long)N, 1.f, ub, h1, dX, ub, c->st);
    launch_lincomb((long long)N, 1.f, ub + N, h2, dX + N, ub + N, c->st);
    std::swap(ua, ub);
  }
  check_launch(c, "deformation map");
  check(c, cudaMemcpyAsync(u, ua, 2 * N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
  if (det) {
    spectral(c, F, SPOP_GRAD, 0.0, ua, 1, 2, gr, 2, nullptr);
    launch_det_grad((long long)N, gr, det, c->st);
    check_launch(c, "det grad y");
  }
}

reg_status reg_deformation_map(reg_ctx* c, const float* v, float* u, float* det) {
  if (!c || !v || !u) return REG_EINVAL;
  if (unaligned({v, u, det})) return reject_unaligned(c);
  return guarded(c, [&] { deformation_map(c, v, u, det); });
}

reg_status reg_transport_rk2a(reg_ctx* c, const float* v, const float* m0, float* m1, int nt) {
  if (!c || !v || !m0 || !m1 || nt < 1 || nt > (1 << 20)) return REG_EINVAL;
  if (unaligned({v, m0, m1})) return reject_unaligned(c);
  return guarded(c, [&] { rk2a_solve(c, v, m0, m1, nt, -1.f); });
}

reg_status reg_adjoint_rk2a(reg_ctx* c, const float* v, const float* lam1, float* lam0, int nt) {
  if (!c || !v || !lam1 || !lam0 || nt < 1 || nt > (1 << 20)) return REG_EINVAL;
  if (unaligned({v, lam1, lam0})) return reject_unaligned(c);
  return guarded(c, [&] { rk2a_solve(c, v, lam1, lam0, nt, 1.f); });
}

reg_status reg_departure_points(reg_ctx* c, const float* v, float* dX, float* dY) {
  if (!c || !v) return REG_EINVAL;
  if (unaligned({v, dX, dY})) return reject_unaligned(c);
  return guarded(c, [&] {
    Level& F = c->fine;
    const float* cv = coefficients(c, F, v, 2, F.c2);
    launch_departure(F.g.n1, F.g.n2, F.ht, v, cv, dX, dY, F.lagrange, c->st);
    check_launch(c, "departure points");
  });
}

reg_status reg_interpolate(reg_ctx* c, const float* u, const float* disp, float* out) {
  if (!c || !u || !disp || !out) return REG_EINVAL;
  if (unaligned({u, disp, out})) return reject_unaligned(c);
  return guarded(c, [&] {
    Level& F = c->fine;
    const float* cu = coefficients(c, F, u, 1, F.coef);
    launch_gather(F.g.n1, F.g.n2, cu, disp, out, 1, 0, F.lagrange, c->st);
    check_launch(c, "interpolate");
  });
}

reg_status reg_spectral(reg_ctx* c, int op, double s, const float* in, float* out) {
  if (!c || !in || !out || in == out) return REG_EINVAL;
  if (unaligned({in, out})) return reject_unaligned(c);
  return guarded(c, [&] {
    Level& F = c->fine;
    switch (op) {
      case REG_SPEC_GRAD: spectral(c, F, SPOP_GRAD, 0.0, in, 1, 1, out, 2, nullptr); break;
      case REG_SPEC_DIV: spectral(c, F, SPOP_DIV, 0.0, in, 2, 1, out, 1, nullptr); break;
      case REG_SPEC_REG: spectral(c, F, SPOP_REGPOW, 1.0, in, 1, 2, out, 1, nullptr); break;
      case REG_SPEC_REGPOW:
        if (s == 1.0) fail(c, REG_EINVAL, "REGPOW with s = 1: use REG_SPEC_REG");
        spectral(c, F, SPOP_REGPOW, s, in, 1, 2, out, 1, nullptr);
        break;
      case REG_SPEC_LOWPASS: spectral(c, F, SPOP_LOWPASS, 0.0, in, 1, 2, out, 1, nullptr); break;
      case REG_SPEC_HIGHPASS: spectral(c, F, SPOP_HIGHPASS, 0.0, in, 1, 2, out, 1, nullptr); break;
      case REG_SPEC_LERAY: spectral(c, F, SPOP_LERAY, 0.0, in, 2, 1, out, 2, nullptr); break;
      case REG_SPEC_REGOP:
        if (c->beta_w > 0.0)
          spectral(c, F, SPOP_REGW, s, in, 2, 1, out, 2, nullptr);
        else
          spectral(c, F, SPOP_REGPOW, s, in, 1, 2, out, 1, nullptr);
        break;
      case REG_SPEC_K:
        if (has_K(c))
          spectral(c, F, K_op(c), 0.0, in, 2, 1, out, 2, nullptr);
        else
          check(c, cudaMemcpyAsync(out, in, 2 * (size_t)F.g.N * sizeof(float), cudaMemcpyDeviceToDevice,
                                   c->st), "copy");
        break;
      case REG_SPEC_PREFILTER:
        if (F.lagrange) fail(c, REG_EINVAL, "PREFILTER needs the spline model");
        coefficients(c, F, in, 1, out);
        break;
      default: fail(c, REG_EINVAL, "unknown spectral op %d", op);
    }
  });
}

reg_status reg_restrict(reg_ctx* c, const float* fine, float* coarse) {
  if (!c || !fine || !coarse) return REG_EINVAL;
  if (unaligned({fine, coarse})) return reject_unaligned(c);
  if (!c->two_level) { c->err = "restriction needs the two-level context"; return REG_ESTATE; }
  return guarded(c, [&] { resample(c, c->fine, c->coarse, SPOP_SCALE, 0.0, fine, 2, coarse, nullptr); });
}

reg_status reg_prolong(reg_ctx* c, const float* coarse, float* fine) {
  if (!c || !fine || !coarse) return REG_EINVAL;
  if (unaligned({fine, coarse})) return reject_unaligned(c);
  if (!c->two_level) { c->err = "prolongation needs the two-level context"; return REG_ESTATE; }
  return guarded(c, [&] { resample(c, c->coarse, c->fine, SPOP_SCALE, 0.0, coarse, 2, fine, nullptr); });
}

reg_status reg_objective_gradient(reg_ctx* c, const float* v, double* J, float* g) {
  if (!c || !v || !J) return REG_EINVAL;
  if (unaligned({v, g})) return reject_unaligned(c);
  return guarded(c, [&] {
    require_images(c);
    *J = objective_gradient(c, v, g);
  });
}

reg_status reg_objective(reg_ctx* c, const float* v, double* J) {
  return reg_objective_gradient(c, v, J, nullptr);
}

// compare v with the cached velocity; rebuild the cache if it differs
static void sync_velocity(reg_ctx* c, const float* v) {
  Level& F = c->fine;
  const long long n = 2 * F.g.N;
  bool differ = true;
  if (F.have_v) {
    check(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st), "memset");
    launch_compare(v, F.v, n, c->dflag, c->st);
    check(c, cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->st), "flag");
    check(c, cudaStreamSynchronize(c->st), "sync");
    differ = (*c->hflag != 0);
  }
  if (differ) set_velocity(c, F, v);
}

reg_status reg_hessian_matvec(reg_ctx* c, const float* v, const float* vt, float* Hvt) {
  if (!c || !v || !vt || !Hvt) return REG_EINVAL;
  if (unaligned({v, vt, Hvt})) return reject_unaligned(c);
  return guarded(c, [&] {
    require_images(c);
    sync_velocity(c, v);
    Level& F = c->fine;
    ensure_G(c, F);
    // the full-Newton matvec reads the adjoint history of this velocity
    if (c->full_newton && !F.have_lam) {
      objective(c, F);
      gradient(c, F, F.w2);
    }
    // repeated calls with the same buffers replay the launch sequence as a
    // CUDA graph, as inside the solver's PCG
    graphed(c, graph_key(c, "mv", vt, Hvt), [&] { hessian_core(c, F, vt, Hvt, false); });
  });
}

reg_status reg_precond_apply(reg_ctx* c, const float* r, float* z) {
  if (!c || !r || !z) return REG_EINVAL;
  if (unaligned({r, z})) return reject_unaligned(c);
  return guarded(c, [&] {
    require_images(c);
    if (!c->fine.have_v) fail(c, REG_ESTATE, "no cached velocity: call reg_objective_gradient first");
    if (c->two_level) {
      if (!c->have_eig) estimate_eigenvalues(c);
      coarse_velocity(c);
      ensure_G(c, c->coarse);
    }
    precond(c, r, z);
  });
}

reg_status reg_kkt_solve(reg_ctx* c, const float* v, const float* rhs, double rtol, int maxit,
                         float* x, reg_info* info) {
  if (!c || !v || !rhs || !x || maxit < 1) return REG_EINVAL;
  if (unaligned({v, rhs, x})) return reject_unaligned(c);
  return guarded(c, [&] {
    require_images(c);
    sync_velocity(c, v);
    c->eta = rtol;
    c->coarse_matvecs = 0;
    const PcgResult r = kkt(c, rhs, rtol, maxit, x);
    if (info) {
      std::memset(info, 0, sizeof *info);
      info->pcg_iters = r.iters;
      info->matvecs = r.matvecs;
      info->coarse_matvecs = c->coarse_matvecs;
      info->gnorm_rel = r.relres;
      info->status = r.negcurv ? REG_ENEGCURV : REG_OK;
    }
  });
}

reg_status reg_eigen_bounds(reg_ctx* c, double* emin, double* emax) {
  if (!c || !emin || !emax) return REG_EINVAL;
  if (!c->two_level) { c->err = "eigenvalue bounds belong to the two-level preconditioner"; return REG_ESTATE; }
  return guarded(c, [&] {
    require_images(c);
    estimate_eigenvalues(c);
    *emin = c->emin;
    *emax = c->emax;
  });
}

reg_status reg_profile_enable(reg_ctx* c, int enable) {
  if (!c) return REG_EINVAL;
  return guarded(c, [&] {
    harvest(c);
    c->prof = enable != 0;
    // events are created here, not while a graph is being captured
    while (c->prof && c->evpool.size() < 16384) {
      cudaEvent_t e;
      check(c, cudaEventCreate(&e), "cudaEventCreate");
      c->evpool.push_back(e);
    }
    for (int l = 0; l < 2; ++l)
      for (int k = 0; k < REG_KC_COUNT; ++k) {
        c->prof_ms[l][k] = 0.0;
        c->prof_bytes[l][k] = 0.0;
        c->prof_n[l][k] = 0;
      }
  });
}

reg_status reg_profile_read(reg_ctx* c, int level, int kclass, double* ms, long long* launches,
                            double* bytes) {
  if (!c || kclass < 0 || kclass >= REG_KC_COUNT || level < 0 || level > 1) return REG_EINVAL;
  return guarded(c, [&] {
    harvest(c);
    if (ms) *ms = c->prof_ms[level][kclass];
    if (launches) *launches = c->prof_n[level][kclass];
    if (bytes) *bytes = c->prof_bytes[level][kclass];
  });
}

long long reg_launch_count(void) { return g_launch_count.load(); }

reg_status reg_step_tiles(const reg_ctx* c, int* tiles) {
  if (!c || !tiles) return REG_EINVAL;
  tiles[0] = c->fine.tile_adj;
  tiles[1] = c->fine.tile_inc;
  tiles[2] = c->two_level ? c->coarse.tile_adj : 0;
  tiles[3] = c->two_level ? c->coarse.tile_inc : 0;
  return REG_OK;
}

reg_status reg_dot(reg_ctx* c, const float* a, const float* b, long long n, double* out) {
  if (!c || !out || n < 0 || (n > 0 && (!a || !b))) return REG_EINVAL;
  if (n == 0) {   // the empty sum (a and b may be NULL)
    *out = 0.0;
    return REG_OK;
  }
  return guarded(c, [&] { *out = dot_sync(c, a, b, n, S_C); });
}

reg_status reg_warm_start(reg_ctx* c, reg_unet* net, float* v, int* accepted) {
  if (!c || !net || !v) return REG_EINVAL;
  if (unaligned({v})) return reject_unaligned(c);
  return guarded(c, [&] {
    require_images(c);
    Level& F = c->fine;
    const int S = reg_unet_size(net);
    int n = F.g.n1, r = 0;
    while (n > S && n % 2 == 0) {
      n /= 2;
      ++r;
    }
    if (F.g.n1 != F.g.n2 || n != S || r > 2)
      fail(c, REG_EINVAL, "warm start needs a square grid of 1, 2 or 4 times the network's size");
    const long long N = F.g.N;
    // m_R, m_T restricted to the network's grid (scratch: F.w1, F.w2)
    const float* mR = F.mR;
    const float* mT = F.mT;
    float* bufR[2] = {F.w1, F.w1 + N / 2};
    float* bufT[2] = {F.w2, F.w2 + N / 2};
    int m = F.g.n1;
    for (int k = 0; k < r; ++k) {
      resample_square(c, m, m / 2, mR, 1, bufR[k & 1]);
      resample_square(c, m, m / 2, mT, 1, bufT[k & 1]);
      mR = bufR[k & 1];
      mT = bufT[k & 1];
      m /= 2;
    }
    float* vs = r == 0 ? v : F.w2 + N;      // 2 S^2 floats
    reg_unet_set_stream(net, c->st);
    const reg_status s = reg_unet_forward(net, 1, nullptr, mR, mT, vs);
    if (s != REG_OK) fail(c, s, "network: %s", reg_unet_last_error(net));
    // prolongation of both velocity components back to the problem grid
    const float* src = vs;
    for (int k = 0; k < r; ++k) {
      float* dst = (k == r - 1) ? v : F.w1 + N;
      resample_square(c, m, 2 * m, src, 2, dst);
      src = dst;
      m *= 2;
    }
    if (c->incompressible) {   // the network's velocity made divergence free
      spectral(c, F, SPOP_LERAY, 0.0, v, 2, 1, F.w1, 2, nullptr);
      check(c, cudaMemcpyAsync(v, F.w1, 2 * N * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
    }
    // accepted only if it lowers the objective below J(0); J(0) comes with
    // the gradient at v = 0 that the solve's relative tolerance needs anyway
    ensure_gref(c);
    const double J1 = objective_gradient(c, v, nullptr);
    const int ok = (J1 < c->J_zero) ? 1 : 0;
    if (!ok) launch_fill(v, 2 * N, 0.f, c->st);
    if (accepted) *accepted = ok;
    check(c, cudaStreamSynchronize(c->st), "warm start");
  });
}

reg_status reg_solve(reg_ctx* c, float* v, double gtol, reg_info* info) {
  if (!c || !v || !(gtol > 0.0)) return REG_EINVAL;
  if (unaligned({v})) return reject_unaligned(c);
  reg_status result = REG_OK;
  reg_info inf;
  std::memset(&inf, 0, sizeof inf);
  const auto t0 = std::chrono::steady_clock::now();
  const reg_status s = guarded(c, [&] {
    require_images(c);
    Level& F = c->fine;
    const long long n = 2 * F.g.N;
    const double hh = F.h1 * F.h2;
    if (c->incompressible) {   // iterates stay divergence free from a projected start
      spectral(c, F, SPOP_LERAY, 0.0, v, 2, 1, c->vt_tmp, 2, nullptr);
      check(c, cudaMemcpyAsync(v, c->vt_tmp, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "copy");
    }
    ensure_gref(c);
    inf.gref_inf = c->gref_inf;
    double J = objective_gradient(c, v, c->gcur);
    inf.J0 = J;
    double rel = 1.0, ginf = 0.0;
    c->coarse_matvecs = 0;
    for (int k = 0;; ++k) {
      ginf = max_abs_sync(c, c->gcur, n, S_GINF);
      if (!std::isfinite(ginf) || !std::isfinite(J)) { result = REG_ENONFINITE; break; }
      rel = ginf / c->gref_inf;
      if (rel <= gtol || ginf <= c->opt.gabs) break;
      if (k == c->opt.max_newton) { result = REG_ENOTCONV; break; }
      const double g2 = std::sqrt(dot_sync(c, c->gcur, c->gcur, n, S_G2));
      c->eta = std::fmin(0.5, g2 / c->gref_2);
      launch_lincomb(n, -1.f, c->gcur, 0.f, nullptr, c->vt_tmp, c->st);   // rhs = -g
      const PcgResult pr = kkt(c, c->vt_tmp, c->eta, c->opt.max_pcg, c->kx);
      inf.pcg_iters += pr.iters;
      inf.matvecs += pr.matvecs;
      const double slope = hh * dot_sync(c, c->gcur, c->kx, n, S_D);
      double alpha = 1.0, Jt = J;
      bool ok = false;
      for (int ls = 0; ls <= c->opt.max_backtracks; ++ls) {
        launch_lincomb(n, 1.f, v, (float)alpha, c->kx, c->vtrial, c->st);
        set_velocity(c, F, c->vtrial);
        Jt = objective(c, F);
        ++inf.line_search_steps;
        if (Jt <= J + c->opt.armijo_c1 * alpha * slope) { ok = true; break; }
        alpha *= 0.5;
      }
      if (!ok) {
        set_velocity(c, F, v);
        objective(c, F);
        result = REG_ELINESEARCH;
        break;
      }
      check(c, cudaMemcpyAsync(v, c->vtrial, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st), "accept");
      J = Jt;
      gradient(c, F, c->gcur);
      ++inf.newton_iters;
    }
    inf.J = J;
    inf.gnorm_rel = rel;
    inf.gnorm_inf = ginf;
    inf.coarse_matvecs = c->coarse_matvecs;
    check(c, cudaStreamSynchronize(c->st), "sync");
  });
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (s != REG_OK) result = s;
  inf.status = result;
  if (info) *info = inf;
  return result;
}

}  // extern "C"
