// Many independent registration problems at once (grids may differ).
//
// A small grid (128^2 .. 512^2) runs each transport step, FFT pass and
// reduction as a kernel that occupies only part of the GPU for a few
// microseconds, and its Newton-Krylov loop waits on the host for every PCG
// scalar. Solving problems one after the other leaves the GPU idle for most
// of that time. The batch gives every problem its own context and CUDA
// stream and drives the solves from a pool of host threads, so that the
// kernels of different problems overlap on the GPU and one problem's host
// round trips hide behind the others' work. Each problem's result is the
// same as solving it alone (same kernels, same order within the problem).
#include <atomic>
#include <chrono>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "reg.h"

struct reg_batch {
  int device = 0;
  std::vector<reg_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<reg_grid> grids;
  std::string err;
};

namespace {

reg_status batch_fail(reg_batch* b, reg_status s, const std::string& msg) {
  b->err = msg;
  return s;
}

}  // namespace

extern "C" {

reg_status reg_batch_create(const reg_grid* grids, int B, int nt, const double* beta,
                            const reg_options* opt, reg_batch** out) {
  if (!out || !grids || !beta || B < 1 || B > 4096) return REG_EINVAL;
  *out = nullptr;
  reg_batch* b = new reg_batch();
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return REG_ECUDA;
  }
  b->grids.assign(grids, grids + B);
  // the problems' kernels run concurrently on one GPU: no context may use
  // the flow kernel, whose blocks wait for each other and need every tile
  // resident at once (two such launches could each hold part of the GPU)
  reg_options o;
  if (opt) o = *opt; else reg_default_options(&o);
  o.flow_matvec = 0;
  for (int i = 0; i < B; ++i) {
    reg_ctx* c = nullptr;
    const reg_status s = reg_create(grids[i], nt, beta[i], &o, &c);
    if (s != REG_OK) {
      reg_batch_destroy(b);
      return s;
    }
    b->ctx.push_back(c);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      reg_batch_destroy(b);
      return REG_ECUDA;
    }
    b->streams.push_back(st);
    reg_set_stream(c, st);
  }
  *out = b;
  return REG_OK;
}

reg_status reg_batch_destroy(reg_batch* b) {
  if (!b) return REG_OK;
  for (size_t i = 0; i < b->ctx.size(); ++i) reg_destroy(b->ctx[i]);
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  delete b;
  return REG_OK;
}

reg_status reg_batch_set_images(reg_batch* b, const float* const* m_R, const float* const* m_T) {
  if (!b || !m_R || !m_T) return REG_EINVAL;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    const reg_status s = reg_set_images(b->ctx[i], m_R[i], m_T[i]);
    if (s != REG_OK)
      return batch_fail(b, s, "problem " + std::to_string(i) + ": " + reg_last_error(b->ctx[i]));
  }
  for (cudaStream_t st : b->streams)
    if (cudaStreamSynchronize(st) != cudaSuccess) return batch_fail(b, REG_ECUDA, "synchronise");
  return REG_OK;
}

reg_status reg_batch_set_beta(reg_batch* b, const double* beta) {
  if (!b || !beta) return REG_EINVAL;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    const reg_status s = reg_set_beta(b->ctx[i], beta[i]);
    if (s != REG_OK) return batch_fail(b, s, "problem " + std::to_string(i));
  }
  return REG_OK;
}

reg_status reg_batch_solve(reg_batch* b, float* const* v, double gtol, int threads,
                           reg_info* infos) {
  if (!b || !v || !(gtol > 0.0)) return REG_EINVAL;
  const int B = (int)b->ctx.size();
  // default: half the host's hardware threads (at least 1, at most B). Each
  // worker alternates between launching and waiting for its problem's
  // scalars; on a 16-core host 8 workers measured fastest (59-60 ms per
  // batch of 64, against 64-70 ms with 32 and 68 ms with 4)
  int T = threads;
  if (T <= 0) {
    const int hc = (int)std::thread::hardware_concurrency();
    T = hc > 1 ? hc / 2 : 1;
  }
  if (T > B) T = B;
  std::vector<reg_info> info(B);
  std::vector<reg_status> st(B, REG_OK);
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(b->device);
    for (int i = next++; i < B; i = next++) st[i] = reg_solve(b->ctx[i], v[i], gtol, &info[i]);
  };
  std::vector<std::thread> pool;
  for (int k = 0; k < T; ++k) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  if (infos) std::memcpy(infos, info.data(), sizeof(reg_info) * B);
  reg_status worst = REG_OK;
  for (int i = 0; i < B; ++i) {
    if (st[i] == REG_OK) continue;
    if (st[i] == REG_ENOTCONV || st[i] == REG_ELINESEARCH) {
      if (worst == REG_OK) worst = st[i];
      continue;
    }
    return batch_fail(b, st[i], "problem " + std::to_string(i) + ": " + reg_last_error(b->ctx[i]));
  }
  return worst;
}

reg_status reg_batch_hessian_matvec(reg_batch* b, const float* const* v, const float* const* vt,
                                    float* const* Hvt) {
  if (!b || !v || !vt || !Hvt) return REG_EINVAL;
  const int B = (int)b->ctx.size();
  const int T = B < 32 ? B : 32;
  std::vector<reg_status> st(B, REG_OK);
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(b->device);
    for (int i = next++; i < B; i = next++) {
      st[i] = reg_hessian_matvec(b->ctx[i], v[i], vt[i], Hvt[i]);
      if (st[i] == REG_OK && cudaStreamSynchronize(b->streams[i]) != cudaSuccess) st[i] = REG_ECUDA;
    }
  };
  std::vector<std::thread> pool;
  for (int k = 0; k < T; ++k) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  for (int i = 0; i < B; ++i)
    if (st[i] != REG_OK)
      return batch_fail(b, st[i], "problem " + std::to_string(i) + ": " + reg_last_error(b->ctx[i]));
  return REG_OK;
}

const char* reg_batch_last_error(const reg_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
