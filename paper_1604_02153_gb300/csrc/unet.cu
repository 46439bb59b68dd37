// Learned warm start: a U-Net that maps (m_R, m_T) to a stationary velocity
// v_0 for the Gauss-Newton-Krylov solve (no counterpart in the paper; the
// solve of §3.4 runs to the same gradient tolerance from v_0 and is the
// arbiter of the result). Forward pass, backward pass and Adam are the
// library's own kernels: every 3x3 convolution, its data gradient and its
// weight gradient are implicit GEMMs on the BF16 tensor cores (mma.sync
// m16n8k16, FP32 accumulation), with activations and activation gradients
// stored as BF16 and master weights, weight gradients and Adam moments in
// FP32.
//
// Architecture: 4 levels with 32, 64, 128, 256 channels, two periodic 3x3
// convolutions + bias + ReLU per level, 2x2 average pooling down, nearest
// 2x upsampling up, skip concatenation [upsampled, encoder output], and a
// last 3x3 convolution to the 2 velocity components (no activation).
//
// Layouts. Activations are NHWC BF16 with a pixel stride `ld` >= channels
// (so a layer can write straight into its slice of a concatenation buffer).
// A layer's device weights are [Coutp][Kp] with k = t * Cin_d + ci (tap
// t = 3a + b of offset (a - 1, b - 1) in (h, w)), Cin_d the input channels
// rounded up to 8, Kp = 9 Cin_d rounded up to 32 and Coutp the output
// channels rounded up to 64; padding entries are zero and stay zero. The
// data-gradient convolution uses the flipped, transposed copy
// Wt[ci][t' * Cout_d + co] = W[co][8 - t'][ci].
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "reg.h"

namespace regnk {
namespace unet {

using bf16 = __nv_bfloat16;
using bf162 = __nv_bfloat162;

// ---------------------------------------------------------------------------
// PTX helpers (sm_80+ forms, valid on sm_103a)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* smem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* smem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}
// D = A (16x16, row) * B (16x8, col) + D, BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// source pixel of tap t for pixel (img, h, w)
__device__ __forceinline__ long long tap_pixel(int img, int h, int w, int t, int H, int W) {
  const int hh = wrap1(h + t / 3 - 1, H), ww = wrap1(w + t % 3 - 1, W);
  return ((long long)img * H + hh) * W + ww;
}

// ---------------------------------------------------------------------------
// Convolution as implicit GEMM: out[p][co] = sum_k A[p][k] Wd[co][k],
// A[p][t * Cin + ci] = in[tap_pixel(p, t)][ci]. Block tile 128 pixels x 64
// output channels, K in chunks of 32 (double-buffered with cp.async), four
// warps of 64 x 32.
constexpr int kCT = 128;
constexpr int BM = 128, BN = 64, BK = 32, PITCH = BK + 8;   // 80-byte smem rows

struct ConvArgs {
  const bf16* in;
  int in_ld, Cin;          // Cin: multiple of 8 (zero channels pad a smaller input)
  int P, H, W;             // P = images * H * W
  const bf16* w;           // [Coutp][Kp]
  int Kp;
  const float* bias;       // [Cout] or null
  int Cout;                // stored output channels (even)
  int Cout_rows;           // weight rows (output channels rounded up to 64)
  void* out;
  int out_ld;
  const bf16* mask;        // optional: zero the output where mask <= 0
  int mask_ld;
  int relu;
};

template <bool OUT_F32>
__global__ void __launch_bounds__(kCT) k_conv(ConvArgs a) {
  pdl_enter();
  __shared__ __align__(16) bf16 As[2][BM * PITCH];
  __shared__ __align__(16) bf16 Bs[2][BN * PITCH];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int p0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int HW = a.H * a.W;
  const int p = p0 + tid;
  const bool pvalid = p < a.P;
  int img = 0, h = 0, w = 0;
  if (pvalid) {
    img = p / HW;
    const int r = p - img * HW;
    h = r / a.W;
    w = r - h * a.W;
  }
  const int nk = a.Kp / BK;

  auto load_stage = [&](int kc, int s) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int k = kc * BK + v * 8;
      const int t = k / a.Cin, ci = k - t * a.Cin;
      const bf16* src = a.in;
      int bytes = 0;
      if (pvalid && t < 9) {
        src = a.in + tap_pixel(img, h, w, t, a.H, a.W) * a.in_ld + ci;
        bytes = 16;
      }
      cp_async16(&As[s][tid * PITCH + v * 8], src, bytes);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int q = tid + i * kCT;
      const int row = q >> 2, v = q & 3;
      cp_async16(&Bs[s][row * PITCH + v * 8], a.w + (long long)(n0 + row) * a.Kp + kc * BK + v * 8, 16);
    }
  };

  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

  load_stage(0, 0);
  cp_async_commit();
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc & 1;
    if (kc + 1 < nk) load_stage(kc + 1, s ^ 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      unsigned af[4][4], bfr[4][2];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
        ldsm_x4(af[mt], &As[s][(wm * 64 + mt * 16 + (lane & 15)) * PITCH + ks * 16 + (lane >> 4) * 8]);
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        unsigned r[4];
        ldsm_x4(r, &Bs[s][(wn * 32 + np * 16 + (lane & 7) + ((lane >> 4) << 3)) * PITCH + ks * 16 +
                          ((lane >> 3) & 1) * 8]);
        bfr[2 * np][0] = r[0];
        bfr[2 * np][1] = r[1];
        bfr[2 * np + 1][0] = r[2];
        bfr[2 * np + 1][1] = r[3];
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt][0], bfr[nt][1]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int pp = p0 + wm * 64 + mt * 16 + (lane >> 2) + half * 8;
      if (pp >= a.P) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int col = n0 + wn * 32 + nt * 8 + 2 * (lane & 3);
        if (col >= a.Cout) continue;
        float x0 = acc[mt][nt][2 * half], x1 = acc[mt][nt][2 * half + 1];
        if (a.bias) {
          x0 += a.bias[col];
          x1 += a.bias[col + 1];
        }
        if (a.relu) {
          x0 = fmaxf(x0, 0.f);
          x1 = fmaxf(x1, 0.f);
        }
        if (a.mask) {
          const bf162 m = *reinterpret_cast<const bf162*>(a.mask + (long long)pp * a.mask_ld + col);
          x0 = __bfloat162float(m.x) > 0.f ? x0 : 0.f;
          x1 = __bfloat162float(m.y) > 0.f ? x1 : 0.f;
        }
        if (OUT_F32) {
          *reinterpret_cast<float2*>(static_cast<float*>(a.out) + (long long)pp * a.out_ld + col) =
              make_float2(x0, x1);
        } else {
          *reinterpret_cast<bf162*>(static_cast<bf16*>(a.out) + (long long)pp * a.out_ld + col) =
              __floats2bfloat162_rn(x0, x1);
        }
      }
    }
}

// ---------------------------------------------------------------------------
// The same convolution on the fifth-generation tensor cores: tcgen05.mma
// (kind::f16, BF16 operands, FP32 accumulator in tensor memory) on a 128 x 64
// or 128 x 128 output tile, one elected thread issuing the MMAs, the operands staged in
// shared memory by all 128 threads (cp.async gathers of the periodic 3x3
// taps), three stages of 64 K entries so that two chunks load while the
// tensor core works on the current one; completion is tracked by an mbarrier per stage
// that tcgen05.commit arrives on. The accumulator (128 lanes x 64 FP32
// columns of tensor memory) is read back with tcgen05.ld by the four warps,
// one pixel row per thread, for the same epilogue as k_conv.
//
// Shared-memory operand layout (no swizzle, K-major): 8 rows x 16 bytes
// "core matrices", 128 bytes each, ordered [row group][K group] with the K
// groups of a row group adjacent: the K-adjacent core matrices are 128 bytes
// apart (leading byte offset), the row-adjacent ones 8 * 128 = 1024 bytes
// apart (stride byte offset). One MMA (K = 16) reads two K-adjacent core
// matrices per row group.
//
// Every wait is bounded: a stage whose MMAs have not completed after
// kTcSpin polls sets *err, the block stops issuing, frees its tensor memory
// and returns.
constexpr int kTcSpin = 1 << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor (no swizzle; version 1 at bits 46-47)
__device__ __forceinline__ unsigned long long umma_sdesc(const void* smem, unsigned lbo,
                                                         unsigned sbo) {
  const unsigned a = smem_u32(smem);
  return (unsigned long long)((a >> 4) & 0x3FFFu) |
         ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28
constexpr unsigned umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) |
         ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(phase)
      : "memory");
  return ok != 0;
}

// bounded wait for the given phase of an mbarrier
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned phase) {
  for (int i = 0; i < kTcSpin; ++i)
    if (mbar_try_wait(b, phase)) return true;
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D (tensor memory) (+)= A (smem) B (smem)^T, issued by one thread
__device__ __forceinline__ void tc_mma(unsigned d_tmem, unsigned long long a, unsigned long long b,
                                       unsigned idesc, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// the mbarrier's arrival once every MMA this thread issued before has completed
__device__ __forceinline__ void tc_commit(unsigned long long* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(b))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Tile of the tcgen05 convolution: 128 pixels x TBN output channels (64 or
// 128), K in chunks of kTcBK = 64 (four MMAs of K = 16), kTcStages chunks in
// flight.
constexpr int kTcBK = 64;
constexpr int kTcStages = 3;
template <int TBN>
constexpr size_t tc_smem() { return sizeof(bf16) * kTcStages * (BM + TBN) * kTcBK; }

// element (row, 8-element K group kv) of a [rows][kTcBK] operand tile in the
// core-matrix layout above
__device__ __forceinline__ int tc_off(int row, int kv) {
  return ((row >> 3) * (kTcBK / 8) + kv) * 64 + (row & 7) * 8;
}

constexpr int kTcThreads = 256;   // two threads per pixel row of the tile

template <bool OUT_F32, int TBN>
__global__ void __launch_bounds__(kTcThreads) k_conv_tc(ConvArgs a, int* __restrict__ err) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  bf16* As = reinterpret_cast<bf16*>(tc_smem_raw);               // kTcStages x BM x kTcBK
  bf16* Bs = As + kTcStages * BM * kTcBK;                         // kTcStages x TBN x kTcBK
  __shared__ __align__(8) unsigned long long bar[kTcStages];
  __shared__ unsigned tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int p0 = blockIdx.x * BM, n0 = blockIdx.y * TBN;
  const int HW = a.H * a.W;
  // loads: pixel row tid % BM, K groups (tid / BM) * 4 .. + 3 of a chunk;
  // epilogue: warp w reads lane quadrant w % 4, column half w / 4
  const int prow = tid % BM, khalf = tid / BM;
  const int p = p0 + prow;
  const bool pvalid = p < a.P;
  int img = 0, h = 0, w = 0;
  if (pvalid) {
    img = p / HW;
    const int r = p - img * HW;
    h = r / a.W;
    w = r - h * a.W;
  }
  const int nk = (a.Kp + kTcBK - 1) / kTcBK;
  const int rows = a.Cout_rows;   // weight rows present (a multiple of 64)
  if (warp == 0) {   // tensor memory for the accumulator (one warp allocates and frees)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"((unsigned)TBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kTcStages; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;

  // K entries at or beyond Kp, and weight rows beyond the stored ones, are
  // zero-filled (cp.async with no source bytes)
  auto load_stage = [&](int kc, int s) {
    bf16* as = As + s * BM * kTcBK;
    bf16* bs = Bs + s * TBN * kTcBK;
#pragma unroll
    for (int vv = 0; vv < kTcBK / 16; ++vv) {
      const int v = khalf * (kTcBK / 16) + vv;
      const int k = kc * kTcBK + v * 8;
      const int t = k / a.Cin, ci = k - t * a.Cin;
      const bf16* src = a.in;
      int bytes = 0;
      if (pvalid && t < 9 && k < a.Kp) {
        src = a.in + tap_pixel(img, h, w, t, a.H, a.W) * a.in_ld + ci;
        bytes = 16;
      }
      cp_async16(&as[tc_off(prow, v)], src, bytes);
    }
#pragma unroll
    for (int i = 0; i < TBN * (kTcBK / 8) / kTcThreads; ++i) {
      const int q = tid + i * kTcThreads;
      const int row = q / (kTcBK / 8), v = q % (kTcBK / 8);
      const int k = kc * kTcBK + v * 8;
      const bool okb = (n0 + row) < rows && k < a.Kp;
      cp_async16(&bs[tc_off(row, v)], okb ? a.w + (long long)(n0 + row) * a.Kp + k : a.w,
                 okb ? 16 : 0);
    }
  };

  constexpr unsigned idesc = umma_idesc_bf16(BM, TBN);
  constexpr unsigned kSbo = (kTcBK / 8) * 128;   // bytes between row-adjacent core matrices
  // stage s holds chunk kc = s (mod kTcStages); the j-th MMA batch reading
  // stage s completes phase j of bar[s]
#pragma unroll
  for (int st = 0; st < kTcStages - 1; ++st) {
    if (st < nk) load_stage(st, st);
    cp_async_commit();
  }
  bool ok = true;
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc % kTcStages;
    cp_async_wait<kTcStages - 2>();   // chunk kc has landed
    // the generic-proxy writes of this stage become visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < kTcBK / 16; ++ks) {
        const unsigned long long ad = umma_sdesc(As + s * BM * kTcBK + ks * 2 * 64, 128, kSbo);
        const unsigned long long bd = umma_sdesc(Bs + s * TBN * kTcBK + ks * 2 * 64, 128, kSbo);
        tc_mma(tmem, ad, bd, idesc, (kc > 0 || ks > 0) ? 1 : 0);
      }
      tc_commit(&bar[s]);
    }
    // refill the stage the previous chunk's MMAs read
    const int kn = kc + kTcStages - 1;
    if (kn < nk) {
      if (kc >= 1) {
        const int sp = (kc - 1) % kTcStages;
        ok = mbar_wait(&bar[sp], (unsigned)(((kc - 1) / kTcStages) & 1));
        if (__syncthreads_or(!ok)) { ok = false; break; }
      }
      load_stage(kn, kn % kTcStages);
    }
    cp_async_commit();
  }
  cp_async_wait<0>();
  // MMAs complete in issue order: the last batch's arrival covers them all
  if (ok) ok = mbar_wait(&bar[(nk - 1) % kTcStages], (unsigned)(((nk - 1) / kTcStages) & 1));
  tc_fence_after();
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    // epilogue: warp w holds pixels p0 + 32 (w % 4) .. + 31 (one per lane) and
    // columns n0 + (w / 4) TBN / 2 .. + TBN / 2 - 1
    const int pp = p0 + (warp & 3) * 32 + (tid & 31);
    const int cbase = (warp >> 2) * (TBN / 2);
#pragma unroll 1
    for (int c = cbase; c < cbase + TBN / 2; c += 16) {
      float x[16];
      tc_ld16(tmem + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)c, x);
      if (pp < a.P) {
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
          const int col = n0 + c + e;
          if (col >= a.Cout) continue;
          float x0 = x[e], x1 = x[e + 1];
          if (a.bias) {
            x0 += a.bias[col];
            x1 += a.bias[col + 1];
          }
          if (a.relu) {
            x0 = fmaxf(x0, 0.f);
            x1 = fmaxf(x1, 0.f);
          }
          if (a.mask) {
            const bf162 m = *reinterpret_cast<const bf162*>(a.mask + (long long)pp * a.mask_ld + col);
            x0 = __bfloat162float(m.x) > 0.f ? x0 : 0.f;
            x1 = __bfloat162float(m.y) > 0.f ? x1 : 0.f;
          }
          if (OUT_F32) {
            *reinterpret_cast<float2*>(static_cast<float*>(a.out) + (long long)pp * a.out_ld + col) =
                make_float2(x0, x1);
          } else {
            *reinterpret_cast<bf162*>(static_cast<bf16*>(a.out) + (long long)pp * a.out_ld + col) =
                __floats2bfloat162_rn(x0, x1);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((unsigned)TBN)
                 : "memory");
}

// ---------------------------------------------------------------------------
// Weight gradient: dW[co][k] += sum_p dz[p][co] A[p][k] over a range of
// pixels per block (FP32 atomics across blocks). Block tile 64 x 64, pixels
// in chunks of 32; both operands are staged pixel-major and read with
// transposing ldmatrix.
constexpr int WPITCH = 64 + 8;   // 144-byte smem rows

struct WgradArgs {
  const bf16* dz;
  int dz_ld, Coutr;        // Coutr: output channels rounded up to 8 (zero beyond Cout)
  const bf16* in;
  int in_ld, Cin;
  int P, H, W;
  int Cout, Kp;
  float* dw;               // [Coutp][Kp]
  int pix_per_block;       // multiple of 32
};

__global__ void __launch_bounds__(kCT) k_wgrad(WgradArgs a) {
  pdl_enter();
  __shared__ __align__(16) bf16 Az[2][32 * WPITCH];
  __shared__ __align__(16) bf16 Bx[2][32 * WPITCH];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int n0 = blockIdx.x * 64, m0 = blockIdx.y * 64;
  const int pb = blockIdx.z * a.pix_per_block;
  const int pe = min(a.P, pb + a.pix_per_block);
  const int HW = a.H * a.W;
  const int nch = (pe - pb + 31) / 32;

  auto load_stage = [&](int c, int s) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int q = tid + i * kCT;       // 0..255: pixel q / 8, vector q % 8
      const int pr = q >> 3, v = q & 7;
      const int p = pb + c * 32 + pr;
      const bool pv = p < pe;
      {
        const int co = m0 + v * 8;
        const bool ok = pv && co < a.Coutr;
        cp_async16(&Az[s][pr * WPITCH + v * 8], ok ? a.dz + (long long)p * a.dz_ld + co : a.dz, ok ? 16 : 0);
      }
      {
        const int k = n0 + v * 8;
        const int t = k / a.Cin, ci = k - t * a.Cin;
        const bf16* src = a.in;
        int bytes = 0;
        if (pv && t < 9) {
          const int img = p / HW, r = p - img * HW, h = r / a.W, w = r - h * a.W;
          src = a.in + tap_pixel(img, h, w, t, a.H, a.W) * a.in_ld + ci;
          bytes = 16;
        }
        cp_async16(&Bx[s][pr * WPITCH + v * 8], src, bytes);
      }
    }
  };

  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

  if (nch > 0) load_stage(0, 0);
  cp_async_commit();
  for (int c = 0; c < nch; ++c) {
    const int s = c & 1;
    if (c + 1 < nch) load_stage(c + 1, s ^ 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      unsigned af[2][4], bfr[4][2];
      const int mi = lane >> 3, r8 = lane & 7;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
        ldsm_x4_t(af[mt], &Az[s][(ks * 16 + r8 + 8 * (mi >> 1)) * WPITCH + wm * 32 + mt * 16 + 8 * (mi & 1)]);
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        unsigned r[4];
        ldsm_x4_t(r, &Bx[s][(ks * 16 + r8 + 8 * (mi & 1)) * WPITCH + wn * 32 + np * 16 + 8 * (mi >> 1)]);
        bfr[2 * np][0] = r[0];
        bfr[2 * np][1] = r[1];
        bfr[2 * np + 1][0] = r[2];
        bfr[2 * np + 1][1] = r[3];
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt][0], bfr[nt][1]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int co = m0 + wm * 32 + mt * 16 + (lane >> 2) + half * 8;
      if (co >= a.Cout) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int k = n0 + wn * 32 + nt * 8 + 2 * (lane & 3);
        if (k >= a.Kp) continue;
        float* d = a.dw + (long long)co * a.Kp + k;
        atomicAdd(d, acc[mt][nt][2 * half]);
        atomicAdd(d + 1, acc[mt][nt][2 * half + 1]);
      }
    }
}

// db[c] += sum over a block of pixels of dz[p][c]
__global__ void k_bias_grad(const bf16* __restrict__ dz, int ld, int C, int P, float* __restrict__ db) {
  pdl_enter();
  const int c = threadIdx.x;
  if (c >= C) return;
  const int p0 = blockIdx.x * 256, p1 = min(P, p0 + 256);
  float s = 0.f;
  for (int p = p0; p < p1; ++p) s += __bfloat162float(dz[(long long)p * ld + c]);
  atomicAdd(db + c, s);
}

// ---------------------------------------------------------------------------
// Pointwise layers (channel vectors of 8 BF16 = 16 bytes; C multiple of 8)

// X0[p] = (m_R, m_T, 0, ..., 0) for image idx[n]
__global__ void k_pack(const float* __restrict__ mR, const float* __restrict__ mT,
                       const int* __restrict__ idx, int B, int HW, bf16* __restrict__ x0) {
  pdl_enter();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)B * HW) return;
  const int n = (int)(p / HW), r = (int)(p - (long long)n * HW);
  const long long src = (long long)(idx ? idx[n] : n) * HW + r;
  bf16 v[8];
  v[0] = __float2bfloat16_rn(mR[src]);
  v[1] = __float2bfloat16_rn(mT[src]);
#pragma unroll
  for (int i = 2; i < 8; ++i) v[i] = __float2bfloat16_rn(0.f);
  *reinterpret_cast<uint4*>(x0 + p * 8) = *reinterpret_cast<uint4*>(v);
}

// out[pc][c] = mean of the 2x2 fine pixels (in: [P][in_ld], C channels)
__global__ void k_pool(const bf16* __restrict__ in, int in_ld, bf16* __restrict__ out, int out_ld,
                       int C, int B, int Hc, int Wc) {
  pdl_enter();
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int cv = C / 8;
  if (q >= (long long)B * Hc * Wc * cv) return;
  const int v = (int)(q % cv);
  const long long pc = q / cv;
  const int n = (int)(pc / (Hc * Wc)), r = (int)(pc - (long long)n * Hc * Wc);
  const int hc = r / Wc, wc = r - hc * Wc;
  const int Wf = 2 * Wc;
  const long long pf = ((long long)n * 2 * Hc + 2 * hc) * Wf + 2 * wc;
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long offs[4] = {pf, pf + 1, pf + Wf, pf + Wf + 1};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint4 raw = *reinterpret_cast<const uint4*>(in + offs[k] * in_ld + v * 8);
    const bf16* e = reinterpret_cast<const bf16*>(&raw);
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] += __bfloat162float(e[i]);
  }
  bf16 o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) o[i] = __float2bfloat16_rn(0.25f * s[i]);
  *reinterpret_cast<uint4*>(out + pc * out_ld + v * 8) = *reinterpret_cast<uint4*>(o);
}

// g[pf][c] = bf16(g[pf][c] + dx[pc][c] / 4), then zeroed where y[pf][c] <= 0
// (g and y are slices of the same concatenation layout, stride ld)
__global__ void k_pool_back_mask(bf16* __restrict__ g, const bf16* __restrict__ y, int ld,
                                 const bf16* __restrict__ dx, int dx_ld, int C, int B, int Hf, int Wf) {
  pdl_enter();
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int cv = C / 8;
  if (q >= (long long)B * Hf * Wf * cv) return;
  const int v = (int)(q % cv);
  const long long pf = q / cv;
  const int n = (int)(pf / (Hf * Wf)), r = (int)(pf - (long long)n * Hf * Wf);
  const int hf = r / Wf, wf = r - hf * Wf;
  const long long pc = ((long long)n * (Hf / 2) + hf / 2) * (Wf / 2) + wf / 2;
  uint4 graw = *reinterpret_cast<const uint4*>(g + pf * ld + v * 8);
  const uint4 yraw = *reinterpret_cast<const uint4*>(y + pf * ld + v * 8);
  const uint4 draw = *reinterpret_cast<const uint4*>(dx + pc * dx_ld + v * 8);
  bf16* ge = reinterpret_cast<bf16*>(&graw);
  const bf16* ye = reinterpret_cast<const bf16*>(&yraw);
  const bf16* de = reinterpret_cast<const bf16*>(&draw);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bf16 s = __float2bfloat16_rn(__bfloat162float(ge[i]) + 0.25f * __bfloat162float(de[i]));
    ge[i] = __bfloat162float(ye[i]) > 0.f ? s : __float2bfloat16_rn(0.f);
  }
  *reinterpret_cast<uint4*>(g + pf * ld + v * 8) = graw;
}

// out[pf][c] = in[pc][c] (nearest 2x), written into a slice with stride out_ld
__global__ void k_upsample(const bf16* __restrict__ in, int in_ld, bf16* __restrict__ out, int out_ld,
                           int C, int B, int Hf, int Wf) {
  pdl_enter();
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int cv = C / 8;
  if (q >= (long long)B * Hf * Wf * cv) return;
  const int v = (int)(q % cv);
  const long long pf = q / cv;
  const int n = (int)(pf / (Hf * Wf)), r = (int)(pf - (long long)n * Hf * Wf);
  const int hf = r / Wf, wf = r - hf * Wf;
  const long long pc = ((long long)n * (Hf / 2) + hf / 2) * (Wf / 2) + wf / 2;
  *reinterpret_cast<uint4*>(out + pf * out_ld + v * 8) =
      *reinterpret_cast<const uint4*>(in + pc * in_ld + v * 8);
}

// dz[pc][c] = (sum of the 2x2 fine gradients g[pf][c]) where y[pc][c] > 0
__global__ void k_upsample_back_mask(const bf16* __restrict__ g, int g_ld, const bf16* __restrict__ y,
                                     int y_ld, bf16* __restrict__ dz, int dz_ld, int C, int B, int Hc,
                                     int Wc) {
  pdl_enter();
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int cv = C / 8;
  if (q >= (long long)B * Hc * Wc * cv) return;
  const int v = (int)(q % cv);
  const long long pc = q / cv;
  const int n = (int)(pc / (Hc * Wc)), r = (int)(pc - (long long)n * Hc * Wc);
  const int hc = r / Wc, wc = r - hc * Wc;
  const int Wf = 2 * Wc;
  const long long pf = ((long long)n * 2 * Hc + 2 * hc) * Wf + 2 * wc;
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long offs[4] = {pf, pf + 1, pf + Wf, pf + Wf + 1};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint4 raw = *reinterpret_cast<const uint4*>(g + offs[k] * g_ld + v * 8);
    const bf16* e = reinterpret_cast<const bf16*>(&raw);
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] += __bfloat162float(e[i]);
  }
  const uint4 yraw = *reinterpret_cast<const uint4*>(y + pc * y_ld + v * 8);
  const bf16* ye = reinterpret_cast<const bf16*>(&yraw);
  bf16 o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) o[i] = __float2bfloat16_rn(__bfloat162float(ye[i]) > 0.f ? s[i] : 0.f);
  *reinterpret_cast<uint4*>(dz + pc * dz_ld + v * 8) = *reinterpret_cast<uint4*>(o);
}

// v[n][c][h][w] = pred[p][c] (c = 0, 1)
__global__ void k_unpack(const float* __restrict__ pred, int B, int HW, float* __restrict__ v) {
  pdl_enter();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)B * HW) return;
  const int n = (int)(p / HW), r = (int)(p - (long long)n * HW);
  const float2 x = *reinterpret_cast<const float2*>(pred + 2 * p);
  v[(2LL * n) * HW + r] = x.x;
  v[(2LL * n + 1) * HW + r] = x.y;
}

// mean squared error against v_target[idx[n]] and its gradient
// dpred[p] = (2 (pred - tgt) / count, 0 x 6) in BF16; loss_sum += sum (pred - tgt)^2
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ tgt,
                      const int* __restrict__ idx, int B, int HW, double inv_count,
                      bf16* __restrict__ dpred, double* __restrict__ loss_sum) {
  pdl_enter();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double e2 = 0.0;
  if (p < (long long)B * HW) {
    const int n = (int)(p / HW), r = (int)(p - (long long)n * HW);
    const long long s = (long long)(idx ? idx[n] : n);
    const float2 x = *reinterpret_cast<const float2*>(pred + 2 * p);
    const float d0 = x.x - tgt[(2 * s) * HW + r], d1 = x.y - tgt[(2 * s + 1) * HW + r];
    e2 = (double)d0 * d0 + (double)d1 * d1;
    bf16 o[8];
    o[0] = __float2bfloat16_rn((float)(2.0 * inv_count) * d0);
    o[1] = __float2bfloat16_rn((float)(2.0 * inv_count) * d1);
#pragma unroll
    for (int i = 2; i < 8; ++i) o[i] = __float2bfloat16_rn(0.f);
    *reinterpret_cast<uint4*>(dpred + p * 8) = *reinterpret_cast<uint4*>(o);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, off);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += ws[i];
    atomicAdd(loss_sum, t);
  }
}

// BF16 device weights (forward and flipped-transposed) from the FP32 master
// [Coutp][Kp]; entries outside the valid (co < Cout, t < 9, ci < Cin) range
// of the master are zero.
__global__ void k_weights_bf16(const float* __restrict__ Wm, int Coutp, int Kp, int Cin_d,
                               int Cout, int Cout_d, int Kpt, bf16* __restrict__ Wb,
                               bf16* __restrict__ Wt) {
  pdl_enter();
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)Coutp * Kp) return;
  const int co = (int)(q / Kp), k = (int)(q - (long long)co * Kp);
  const bf16 b = __float2bfloat16_rn(Wm[q]);
  Wb[q] = b;
  const int t = k / Cin_d, ci = k - t * Cin_d;
  if (Wt && co < Cout && t < 9) Wt[(long long)ci * Kpt + (8 - t) * Cout_d + co] = b;
}

// Adam (bias-corrected); c1 = 1 / (1 - beta1^step), c2 = 1 / (1 - beta2^step)
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  pdl_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// ---------------------------------------------------------------------------
// Host side

struct LayerDef {
  const char* name;
  int cin, cout, relu;
};
constexpr LayerDef kLayers[] = {
    {"enc0a", 2, 32, 1},    {"enc0b", 32, 32, 1},   {"enc1a", 32, 64, 1},  {"enc1b", 64, 64, 1},
    {"enc2a", 64, 128, 1},  {"enc2b", 128, 128, 1}, {"enc3a", 128, 256, 1}, {"enc3b", 256, 256, 1},
    {"dec2a", 384, 128, 1}, {"dec2b", 128, 128, 1}, {"dec1a", 192, 64, 1}, {"dec1b", 64, 64, 1},
    {"dec0a", 96, 32, 1},   {"dec0b", 32, 32, 1},   {"out", 32, 2, 0}};
constexpr int kNL = 15;
enum { E0A, E0B, E1A, E1B, E2A, E2B, E3A, E3B, D2A, D2B, D1A, D1B, D0A, D0B, OUT };

inline int up8(int x) { return (x + 7) / 8 * 8; }
inline int up32(int x) { return (x + 31) / 32 * 32; }
inline int up64(int x) { return (x + 63) / 64 * 64; }

struct Layer {
  int cin, cout, relu;
  int cin_d, cout_d, coutp, kp;     // forward GEMM
  int cinp, kpt;                    // data-gradient GEMM: rows cinp (= up64(cin)), K kpt
  float *w, *b, *gw, *gb, *mw, *vw, *mb, *vb;   // FP32 master, gradients, Adam moments
  bf16 *wb, *wt;
};

struct Act {            // an activation tensor [P][ld] (or a slice of one)
  bf16* p = nullptr;
  int ld = 0;
};

}  // namespace unet
}  // namespace regnk

using namespace regnk;
using namespace regnk::unet;

struct reg_unet {
  int size = 0, bmax = 0;
  int device = 0;
  cudaStream_t st = nullptr;
  Layer L[kNL];
  long long step = 0;
  std::string err;
  std::vector<void*> allocs;
  // activations (level l: S_l = size >> l)
  Act x0, e0a, cat0, d0a, d0b, x1, e1a, cat1, d1a, d1b, x2, e2a, cat2, d2a, d2b, x3, e3a, e3b;
  float* pred = nullptr;
  // activation gradients
  Act g_pred, g_d0b, g_d0a, g_cat0, g_e0a, g_x1, g_d1b, g_d1a, g_cat1, g_e1a, g_x2, g_d2b, g_d2a,
      g_cat2, g_e2a, g_x3, g_e3b, g_e3a;
  double* loss = nullptr;
  int conv_path = 0;       // 0: mma.sync convolutions, 1: tcgen05 (tensor memory)
  int* derr = nullptr;     // set by a tcgen05 convolution whose bounded wait ran out
};

namespace {

struct UnetError {
  reg_status s;
};

void ucheck(reg_unet* u, cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    u->err = std::string(what) + ": " + cudaGetErrorString(e);
    throw UnetError{REG_ECUDA};
  }
}

template <typename T>
T* ualloc(reg_unet* u, size_t count) {
  void* p = nullptr;
  ucheck(u, cudaMalloc(&p, count * sizeof(T) + 16), "cudaMalloc");
  u->allocs.push_back(p);
  ucheck(u, cudaMemset(p, 0, count * sizeof(T) + 16), "cudaMemset");
  return static_cast<T*>(p);
}

Act act(reg_unet* u, long long P, int C) {
  Act a;
  a.p = ualloc<bf16>(u, (size_t)P * C);
  a.ld = C;
  return a;
}
Act slice(const Act& a, int c0) { return Act{a.p + c0, a.ld}; }

unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

void conv(reg_unet* u, const Layer& l, const Act& in, int cin, long long P, int S, void* out,
          int out_ld, bool out_f32, bool data_grad, const Act* mask) {
  ConvArgs a{};
  a.in = in.p;
  a.in_ld = in.ld;
  a.P = (int)P;
  a.H = a.W = S;
  if (!data_grad) {
    a.Cin = l.cin_d;
    a.w = l.wb;
    a.Kp = l.kp;
    a.bias = l.b;
    a.Cout = l.cout;
    a.relu = l.relu;
  } else {
    a.Cin = l.cout_d;
    a.w = l.wt;
    a.Kp = l.kpt;
    a.bias = nullptr;
    a.Cout = l.cin;
    a.relu = 0;
  }
  (void)cin;
  a.out = out;
  a.out_ld = out_ld;
  a.mask = mask ? mask->p : nullptr;
  a.mask_ld = mask ? mask->ld : 0;
  const int rows = data_grad ? l.cinp : l.coutp;
  a.Cout_rows = rows;
  const dim3 grid(nblk(P, BM), rows / BN);
  if (u->conv_path == 1) {   // 128-channel tiles where there are 128 or more rows
    if (rows >= 128) {
      const dim3 g2(nblk(P, BM), (rows + 127) / 128);
      if (out_f32)
        launch_k(k_conv_tc<true, 128>, g2, dim3(kTcThreads), tc_smem<128>(), u->st, a, u->derr);
      else
        launch_k(k_conv_tc<false, 128>, g2, dim3(kTcThreads), tc_smem<128>(), u->st, a, u->derr);
    } else {
      if (out_f32)
        launch_k(k_conv_tc<true, 64>, grid, dim3(kTcThreads), tc_smem<64>(), u->st, a, u->derr);
      else
        launch_k(k_conv_tc<false, 64>, grid, dim3(kTcThreads), tc_smem<64>(), u->st, a, u->derr);
    }
    return;
  }
  if (out_f32)
    launch_k(k_conv<true>, grid, dim3(kCT), 0, u->st, a);
  else
    launch_k(k_conv<false>, grid, dim3(kCT), 0, u->st, a);
}

// With the tcgen05 convolutions: synchronises and reports a convolution
// whose bounded wait ran out (REG_ETIMEOUT; the flag is cleared).
void check_tc(reg_unet* u) {
  if (u->conv_path != 1) return;
  int e = 0;
  ucheck(u, cudaMemcpyAsync(&e, u->derr, sizeof(int), cudaMemcpyDeviceToHost, u->st), "error flag");
  ucheck(u, cudaStreamSynchronize(u->st), "error flag");
  if (e) {
    cudaMemsetAsync(u->derr, 0, sizeof(int), u->st);
    cudaStreamSynchronize(u->st);
    u->err = "a tcgen05 convolution gave up waiting for its MMAs";
    throw UnetError{REG_ETIMEOUT};
  }
}

void wgrad(reg_unet* u, const Layer& l, const Act& dz, const Act& in, long long P, int S) {
  WgradArgs a{};
  a.dz = dz.p;
  a.dz_ld = dz.ld;
  a.Coutr = l.cout_d;
  a.in = in.p;
  a.in_ld = in.ld;
  a.Cin = l.cin_d;
  a.P = (int)P;
  a.H = a.W = S;
  a.Cout = l.cout;
  a.Kp = l.kp;
  a.dw = l.gw;
  // about 4 blocks per SM for the smallest layers, at least 32 pixels each
  const long long tiles = (long long)nblk(l.kp, 64) * (l.coutp / 64);
  long long splits = (4 * 152 + tiles - 1) / tiles;
  long long ppb = (P + splits - 1) / splits;
  ppb = ((ppb + 31) / 32) * 32;
  if (ppb < 1024 && P >= 1024) ppb = 1024;
  a.pix_per_block = (int)ppb;
  const dim3 grid(nblk(l.kp, 64), l.coutp / 64, nblk(P, (int)ppb));
  launch_k(k_wgrad, grid, dim3(kCT), 0, u->st, a);
  launch_k(k_bias_grad, dim3(nblk(P, 256)), dim3(256), 0, u->st, (const bf16*)dz.p, dz.ld, l.cout,
           (int)P, l.gb);
}

void pool(reg_unet* u, const Act& in, const Act& out, int C, int B, int Sc) {
  const long long n = (long long)B * Sc * Sc * (C / 8);
  launch_k(k_pool, dim3(nblk(n, 256)), dim3(256), 0, u->st, (const bf16*)in.p, in.ld, out.p, out.ld, C,
           B, Sc, Sc);
}

void upsample(reg_unet* u, const Act& in, const Act& out, int C, int B, int Sf) {
  const long long n = (long long)B * Sf * Sf * (C / 8);
  launch_k(k_upsample, dim3(nblk(n, 256)), dim3(256), 0, u->st, (const bf16*)in.p, in.ld, out.p,
           out.ld, C, B, Sf, Sf);
}

void refresh_bf16(reg_unet* u, int i) {
  Layer& l = u->L[i];
  const long long n = (long long)l.coutp * l.kp;
  launch_k(k_weights_bf16, dim3(nblk(n, 256)), dim3(256), 0, u->st, (const float*)l.w, l.coutp, l.kp,
           l.cin_d, l.cout, l.cout_d, l.kpt, l.wb, l.wt);
}

void forward(reg_unet* u, int B, const int* idx, const float* mR, const float* mT) {
  const int S0 = u->size, S1 = S0 / 2, S2 = S0 / 4, S3 = S0 / 8;
  const long long P0 = (long long)B * S0 * S0, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  Layer* L = u->L;
  launch_k(k_pack, dim3(nblk(P0, 256)), dim3(256), 0, u->st, mR, mT, idx, B, S0 * S0, u->x0.p);
  conv(u, L[E0A], u->x0, 8, P0, S0, u->e0a.p, u->e0a.ld, false, false, nullptr);
  const Act e0b = slice(u->cat0, 64);
  conv(u, L[E0B], u->e0a, 32, P0, S0, e0b.p, e0b.ld, false, false, nullptr);
  pool(u, e0b, u->x1, 32, B, S1);
  conv(u, L[E1A], u->x1, 32, P1, S1, u->e1a.p, u->e1a.ld, false, false, nullptr);
  const Act e1b = slice(u->cat1, 128);
  conv(u, L[E1B], u->e1a, 64, P1, S1, e1b.p, e1b.ld, false, false, nullptr);
  pool(u, e1b, u->x2, 64, B, S2);
  conv(u, L[E2A], u->x2, 64, P2, S2, u->e2a.p, u->e2a.ld, false, false, nullptr);
  const Act e2b = slice(u->cat2, 256);
  conv(u, L[E2B], u->e2a, 128, P2, S2, e2b.p, e2b.ld, false, false, nullptr);
  pool(u, e2b, u->x3, 128, B, S3);
  conv(u, L[E3A], u->x3, 128, P3, S3, u->e3a.p, u->e3a.ld, false, false, nullptr);
  conv(u, L[E3B], u->e3a, 256, P3, S3, u->e3b.p, u->e3b.ld, false, false, nullptr);
  upsample(u, u->e3b, u->cat2, 256, B, S2);
  conv(u, L[D2A], u->cat2, 384, P2, S2, u->d2a.p, u->d2a.ld, false, false, nullptr);
  conv(u, L[D2B], u->d2a, 128, P2, S2, u->d2b.p, u->d2b.ld, false, false, nullptr);
  upsample(u, u->d2b, u->cat1, 128, B, S1);
  conv(u, L[D1A], u->cat1, 192, P1, S1, u->d1a.p, u->d1a.ld, false, false, nullptr);
  conv(u, L[D1B], u->d1a, 64, P1, S1, u->d1b.p, u->d1b.ld, false, false, nullptr);
  upsample(u, u->d1b, u->cat0, 64, B, S0);
  conv(u, L[D0A], u->cat0, 96, P0, S0, u->d0a.p, u->d0a.ld, false, false, nullptr);
  conv(u, L[D0B], u->d0a, 32, P0, S0, u->d0b.p, u->d0b.ld, false, false, nullptr);
  conv(u, L[OUT], u->d0b, 32, P0, S0, u->pred, 2, true, false, nullptr);
}

void zero_grads(reg_unet* u) {
  for (int i = 0; i < kNL; ++i) {
    Layer& l = u->L[i];
    ucheck(u, cudaMemsetAsync(l.gw, 0, sizeof(float) * (size_t)l.coutp * l.kp, u->st), "memset");
    ucheck(u, cudaMemsetAsync(l.gb, 0, sizeof(float) * (size_t)l.cout, u->st), "memset");
  }
}

// loss and gradients for the batch whose forward pass ran last
void backward(reg_unet* u, int B, const int* idx, const float* vt) {
  const int S0 = u->size, S1 = S0 / 2, S2 = S0 / 4, S3 = S0 / 8;
  const long long P0 = (long long)B * S0 * S0, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  Layer* L = u->L;
  ucheck(u, cudaMemsetAsync(u->loss, 0, sizeof(double), u->st), "memset");
  launch_k(k_mse, dim3(nblk(P0, 256)), dim3(256), 0, u->st, (const float*)u->pred, vt, idx, B, S0 * S0,
           1.0 / (2.0 * (double)P0), u->g_pred.p, u->loss);
  zero_grads(u);
  // out
  wgrad(u, L[OUT], u->g_pred, u->d0b, P0, S0);
  conv(u, L[OUT], u->g_pred, 8, P0, S0, u->g_d0b.p, u->g_d0b.ld, false, true, &u->d0b);
  // dec0
  wgrad(u, L[D0B], u->g_d0b, u->d0a, P0, S0);
  conv(u, L[D0B], u->g_d0b, 32, P0, S0, u->g_d0a.p, u->g_d0a.ld, false, true, &u->d0a);
  wgrad(u, L[D0A], u->g_d0a, u->cat0, P0, S0);
  conv(u, L[D0A], u->g_d0a, 32, P0, S0, u->g_cat0.p, u->g_cat0.ld, false, true, nullptr);
  {
    const long long n = (long long)B * S1 * S1 * (64 / 8);
    launch_k(k_upsample_back_mask, dim3(nblk(n, 256)), dim3(256), 0, u->st, (const bf16*)u->g_cat0.p,
             u->g_cat0.ld, (const bf16*)u->d1b.p, u->d1b.ld, u->g_d1b.p, u->g_d1b.ld, 64, B, S1, S1);
  }
  // dec1
  wgrad(u, L[D1B], u->g_d1b, u->d1a, P1, S1);
  conv(u, L[D1B], u->g_d1b, 64, P1, S1, u->g_d1a.p, u->g_d1a.ld, false, true, &u->d1a);
  wgrad(u, L[D1A], u->g_d1a, u->cat1, P1, S1);
  conv(u, L[D1A], u->g_d1a, 64, P1, S1, u->g_cat1.p, u->g_cat1.ld, false, true, nullptr);
  {
    const long long n = (long long)B * S2 * S2 * (128 / 8);
    launch_k(k_upsample_back_mask, dim3(nblk(n, 256)), dim3(256), 0, u->st, (const bf16*)u->g_cat1.p,
             u->g_cat1.ld, (const bf16*)u->d2b.p, u->d2b.ld, u->g_d2b.p, u->g_d2b.ld, 128, B, S2, S2);
  }
  // dec2
  wgrad(u, L[D2B], u->g_d2b, u->d2a, P2, S2);
  conv(u, L[D2B], u->g_d2b, 128, P2, S2, u->g_d2a.p, u->g_d2a.ld, false, true, &u->d2a);
  wgrad(u, L[D2A], u->g_d2a, u->cat2, P2, S2);
  conv(u, L[D2A], u->g_d2a, 128, P2, S2, u->g_cat2.p, u->g_cat2.ld, false, true, nullptr);
  {
    const long long n = (long long)B * S3 * S3 * (256 / 8);
    launch_k(k_upsample_back_mask, dim3(nblk(n, 256)), dim3(256), 0, u->st, (const bf16*)u->g_cat2.p,
             u->g_cat2.ld, (const bf16*)u->e3b.p, u->e3b.ld, u->g_e3b.p, u->g_e3b.ld, 256, B, S3, S3);
  }
  // enc3
  wgrad(u, L[E3B], u->g_e3b, u->e3a, P3, S3);
  conv(u, L[E3B], u->g_e3b, 256, P3, S3, u->g_e3a.p, u->g_e3a.ld, false, true, &u->e3a);
  wgrad(u, L[E3A], u->g_e3a, u->x3, P3, S3);
  conv(u, L[E3A], u->g_e3a, 256, P3, S3, u->g_x3.p, u->g_x3.ld, false, true, nullptr);
  // enc2: skip gradient (slice of g_cat2) + pooled gradient, masked
  const Act ge2b = slice(u->g_cat2, 256), e2b = slice(u->cat2, 256);
  {
    const long long n = (long long)B * S2 * S2 * (128 / 8);
    launch_k(k_pool_back_mask, dim3(nblk(n, 256)), dim3(256), 0, u->st, ge2b.p, (const bf16*)e2b.p,
             ge2b.ld, (const bf16*)u->g_x3.p, u->g_x3.ld, 128, B, S2, S2);
  }
  wgrad(u, L[E2B], ge2b, u->e2a, P2, S2);
  conv(u, L[E2B], ge2b, 128, P2, S2, u->g_e2a.p, u->g_e2a.ld, false, true, &u->e2a);
  wgrad(u, L[E2A], u->g_e2a, u->x2, P2, S2);
  conv(u, L[E2A], u->g_e2a, 128, P2, S2, u->g_x2.p, u->g_x2.ld, false, true, nullptr);
  // enc1
  const Act ge1b = slice(u->g_cat1, 128), e1b = slice(u->cat1, 128);
  {
    const long long n = (long long)B * S1 * S1 * (64 / 8);
    launch_k(k_pool_back_mask, dim3(nblk(n, 256)), dim3(256), 0, u->st, ge1b.p, (const bf16*)e1b.p,
             ge1b.ld, (const bf16*)u->g_x2.p, u->g_x2.ld, 64, B, S1, S1);
  }
  wgrad(u, L[E1B], ge1b, u->e1a, P1, S1);
  conv(u, L[E1B], ge1b, 64, P1, S1, u->g_e1a.p, u->g_e1a.ld, false, true, &u->e1a);
  wgrad(u, L[E1A], u->g_e1a, u->x1, P1, S1);
  conv(u, L[E1A], u->g_e1a, 64, P1, S1, u->g_x1.p, u->g_x1.ld, false, true, nullptr);
  // enc0
  const Act ge0b = slice(u->g_cat0, 64), e0b = slice(u->cat0, 64);
  {
    const long long n = (long long)B * S0 * S0 * (32 / 8);
    launch_k(k_pool_back_mask, dim3(nblk(n, 256)), dim3(256), 0, u->st, ge0b.p, (const bf16*)e0b.p,
             ge0b.ld, (const bf16*)u->g_x1.p, u->g_x1.ld, 32, B, S0, S0);
  }
  wgrad(u, L[E0B], ge0b, u->e0a, P0, S0);
  conv(u, L[E0B], ge0b, 32, P0, S0, u->g_e0a.p, u->g_e0a.ld, false, true, &u->e0a);
  wgrad(u, L[E0A], u->g_e0a, u->x0, P0, S0);
}

void adam(reg_unet* u, float lr) {
  ++u->step;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)u->step)));
  const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)u->step)));
  for (int i = 0; i < kNL; ++i) {
    Layer& l = u->L[i];
    const long long nw = (long long)l.coutp * l.kp;
    launch_k(k_adam, dim3(nblk(nw, 256)), dim3(256), 0, u->st, l.w, (const float*)l.gw, l.mw, l.vw, nw, lr,
             b1, b2, eps, c1, c2);
    launch_k(k_adam, dim3(nblk(l.cout, 256)), dim3(256), 0, u->st, l.b, (const float*)l.gb, l.mb, l.vb,
             (long long)l.cout, lr, b1, b2, eps, c1, c2);
    refresh_bf16(u, i);
  }
}

template <typename F>
reg_status uguard(reg_unet* u, F body) {
  if (!u) return REG_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != u->device) cudaSetDevice(u->device);
  reg_status s = REG_OK;
  try {
    body();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      u->err = std::string("CUDA: ") + cudaGetErrorString(e);
      s = REG_ECUDA;
    }
  } catch (const UnetError& e) {
    s = e.s;
  }
  if (prev != u->device) cudaSetDevice(prev);
  return s;
}

bool batch_ok(const reg_unet* u, int B) { return u && B >= 1 && B <= u->bmax; }

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

long long reg_unet_param_count(void) {
  long long n = 0;
  for (const auto& d : kLayers) n += (long long)d.cout * 9 * d.cin + d.cout;
  return n;
}

reg_status reg_unet_create(int size, int batch_max, reg_unet** out) {
  if (!out) return REG_EINVAL;
  *out = nullptr;
  if (size < 32 || size > 1024 || size % 32 != 0 || batch_max < 1 ||
      (long long)batch_max * size * size > (1LL << 26))
    return REG_EINVAL;
  reg_unet* u = new reg_unet();
  u->size = size;
  u->bmax = batch_max;
  if (cudaGetDevice(&u->device) != cudaSuccess) {
    delete u;
    return REG_ECUDA;
  }
  const reg_status s = uguard(u, [&] {
    for (int i = 0; i < kNL; ++i) {
      Layer& l = u->L[i];
      l.cin = kLayers[i].cin;
      l.cout = kLayers[i].cout;
      l.relu = kLayers[i].relu;
      l.cin_d = up8(l.cin);
      l.cout_d = up8(l.cout);
      l.coutp = up64(l.cout);
      l.kp = up32(9 * l.cin_d);
      l.cinp = up64(l.cin);
      l.kpt = up32(9 * l.cout_d);
      const size_t nw = (size_t)l.coutp * l.kp;
      l.w = ualloc<float>(u, nw);
      l.gw = ualloc<float>(u, nw);
      l.mw = ualloc<float>(u, nw);
      l.vw = ualloc<float>(u, nw);
      l.b = ualloc<float>(u, l.cout);
      l.gb = ualloc<float>(u, l.cout);
      l.mb = ualloc<float>(u, l.cout);
      l.vb = ualloc<float>(u, l.cout);
      l.wb = ualloc<bf16>(u, nw);
      l.wt = ualloc<bf16>(u, (size_t)l.cinp * l.kpt);
    }
    const long long P0 = (long long)batch_max * size * size, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
    u->x0 = act(u, P0, 8);
    u->e0a = act(u, P0, 32);
    u->cat0 = act(u, P0, 96);
    u->d0a = act(u, P0, 32);
    u->d0b = act(u, P0, 32);
    u->x1 = act(u, P1, 32);
    u->e1a = act(u, P1, 64);
    u->cat1 = act(u, P1, 192);
    u->d1a = act(u, P1, 64);
    u->d1b = act(u, P1, 64);
    u->x2 = act(u, P2, 64);
    u->e2a = act(u, P2, 128);
    u->cat2 = act(u, P2, 384);
    u->d2a = act(u, P2, 128);
    u->d2b = act(u, P2, 128);
    u->x3 = act(u, P3, 128);
    u->e3a = act(u, P3, 256);
    u->e3b = act(u, P3, 256);
    u->pred = ualloc<float>(u, (size_t)P0 * 2);
    u->g_pred = act(u, P0, 8);
    u->g_d0b = act(u, P0, 32);
    u->g_d0a = act(u, P0, 32);
    u->g_cat0 = act(u, P0, 96);
    u->g_e0a = act(u, P0, 32);
    u->g_x1 = act(u, P1, 32);
    u->g_d1b = act(u, P1, 64);
    u->g_d1a = act(u, P1, 64);
    u->g_cat1 = act(u, P1, 192);
    u->g_e1a = act(u, P1, 64);
    u->g_x2 = act(u, P2, 64);
    u->g_d2b = act(u, P2, 128);
    u->g_d2a = act(u, P2, 128);
    u->g_cat2 = act(u, P2, 384);
    u->g_e2a = act(u, P2, 128);
    u->g_x3 = act(u, P3, 128);
    u->g_e3b = act(u, P3, 256);
    u->g_e3a = act(u, P3, 256);
    u->loss = ualloc<double>(u, 1);
    u->derr = ualloc<int>(u, 1);
    // the tcgen05 convolutions' operand stages (72 KB and 96 KB of dynamic
    // shared memory)
    ucheck(u, cudaFuncSetAttribute(k_conv_tc<true, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)tc_smem<64>()), "shared memory limit");
    ucheck(u, cudaFuncSetAttribute(k_conv_tc<false, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)tc_smem<64>()), "shared memory limit");
    ucheck(u, cudaFuncSetAttribute(k_conv_tc<true, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)tc_smem<128>()), "shared memory limit");
    ucheck(u, cudaFuncSetAttribute(k_conv_tc<false, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)tc_smem<128>()), "shared memory limit");
    ucheck(u, cudaDeviceSynchronize(), "allocate");
  });
  if (s != REG_OK) {
    reg_unet_destroy(u);
    return s;
  }
  *out = u;
  return REG_OK;
}

reg_status reg_unet_destroy(reg_unet* u) {
  if (!u) return REG_OK;
  if (u->st) cudaStreamSynchronize(u->st);
  for (void* p : u->allocs) cudaFree(p);
  delete u;
  return REG_OK;
}

int reg_unet_size(const reg_unet* u) { return u ? u->size : 0; }

reg_status reg_unet_set_stream(reg_unet* u, void* stream) {
  if (!u) return REG_EINVAL;
  u->st = static_cast<cudaStream_t>(stream);
  return REG_OK;
}

reg_status reg_unet_set_params(reg_unet* u, const float* host) {
  if (!u || !host) return REG_EINVAL;
  return uguard(u, [&] {
    const float* src = host;
    for (int i = 0; i < kNL; ++i) {
      Layer& l = u->L[i];
      std::vector<float> wd((size_t)l.coutp * l.kp, 0.f);
      for (int co = 0; co < l.cout; ++co)
        for (int t = 0; t < 9; ++t)
          for (int ci = 0; ci < l.cin; ++ci)
            wd[(size_t)co * l.kp + t * l.cin_d + ci] = src[((size_t)co * 9 + t) * l.cin + ci];
      src += (size_t)l.cout * 9 * l.cin;
      ucheck(u, cudaMemcpyAsync(l.w, wd.data(), wd.size() * sizeof(float), cudaMemcpyHostToDevice, u->st),
             "copy weights");
      ucheck(u, cudaMemcpyAsync(l.b, src, l.cout * sizeof(float), cudaMemcpyHostToDevice, u->st),
             "copy bias");
      src += l.cout;
      ucheck(u, cudaMemsetAsync(l.mw, 0, wd.size() * sizeof(float), u->st), "memset");
      ucheck(u, cudaMemsetAsync(l.vw, 0, wd.size() * sizeof(float), u->st), "memset");
      ucheck(u, cudaMemsetAsync(l.mb, 0, l.cout * sizeof(float), u->st), "memset");
      ucheck(u, cudaMemsetAsync(l.vb, 0, l.cout * sizeof(float), u->st), "memset");
      refresh_bf16(u, i);
      ucheck(u, cudaStreamSynchronize(u->st), "set params");   // wd is a host temporary
    }
    u->step = 0;
  });
}

static void read_layered(reg_unet* u, bool grads, float* host) {
  float* dst = host;
  for (int i = 0; i < kNL; ++i) {
    Layer& l = u->L[i];
    std::vector<float> wd((size_t)l.coutp * l.kp);
    ucheck(u, cudaMemcpyAsync(wd.data(), grads ? l.gw : l.w, wd.size() * sizeof(float),
                              cudaMemcpyDeviceToHost, u->st), "read weights");
    ucheck(u, cudaMemcpyAsync(dst + (size_t)l.cout * 9 * l.cin, grads ? l.gb : l.b, l.cout * sizeof(float),
                              cudaMemcpyDeviceToHost, u->st), "read bias");
    ucheck(u, cudaStreamSynchronize(u->st), "read");
    for (int co = 0; co < l.cout; ++co)
      for (int t = 0; t < 9; ++t)
        for (int ci = 0; ci < l.cin; ++ci)
          dst[((size_t)co * 9 + t) * l.cin + ci] = wd[(size_t)co * l.kp + t * l.cin_d + ci];
    dst += (size_t)l.cout * 9 * l.cin + l.cout;
  }
}

reg_status reg_unet_get_params(reg_unet* u, float* host) {
  if (!u || !host) return REG_EINVAL;
  return uguard(u, [&] { read_layered(u, false, host); });
}

reg_status reg_unet_forward(reg_unet* u, int B, const int* idx, const float* mR, const float* mT,
                            float* v) {
  if (!batch_ok(u, B) || !mR || !mT || !v) return REG_EINVAL;
  if (!al16(mR) || !al16(mT) || !al16(v)) return REG_EINVAL;
  return uguard(u, [&] {
    forward(u, B, idx, mR, mT);
    const long long P0 = (long long)B * u->size * u->size;
    launch_k(k_unpack, dim3(nblk(P0, 256)), dim3(256), 0, u->st, (const float*)u->pred, B,
             u->size * u->size, v);
    check_tc(u);
  });
}

reg_status reg_unet_gradients(reg_unet* u, int B, const int* idx, const float* mR, const float* mT,
                              const float* v_target, float* host_grad, double* loss) {
  if (!batch_ok(u, B) || !mR || !mT || !v_target) return REG_EINVAL;
  if (!al16(mR) || !al16(mT) || !al16(v_target)) return REG_EINVAL;
  return uguard(u, [&] {
    forward(u, B, idx, mR, mT);
    backward(u, B, idx, v_target);
    check_tc(u);
    if (loss) {
      double s = 0.0;
      ucheck(u, cudaMemcpyAsync(&s, u->loss, sizeof(double), cudaMemcpyDeviceToHost, u->st), "loss");
      ucheck(u, cudaStreamSynchronize(u->st), "loss");
      *loss = s / (2.0 * (double)B * u->size * u->size);
    }
    if (host_grad) read_layered(u, true, host_grad);
  });
}

reg_status reg_unet_train_step(reg_unet* u, int B, const int* idx, const float* mR, const float* mT,
                               const float* v_target, float lr, double* loss) {
  if (!batch_ok(u, B) || !mR || !mT || !v_target || !(lr > 0.f)) return REG_EINVAL;
  if (!al16(mR) || !al16(mT) || !al16(v_target)) return REG_EINVAL;
  return uguard(u, [&] {
    forward(u, B, idx, mR, mT);
    backward(u, B, idx, v_target);
    check_tc(u);
    adam(u, lr);
    if (loss) {
      double s = 0.0;
      ucheck(u, cudaMemcpyAsync(&s, u->loss, sizeof(double), cudaMemcpyDeviceToHost, u->st), "loss");
      ucheck(u, cudaStreamSynchronize(u->st), "loss");
      *loss = s / (2.0 * (double)B * u->size * u->size);
    }
  });
}

reg_status reg_unet_set_conv_path(reg_unet* u, int path) {
  if (!u || (path != 0 && path != 1)) return REG_EINVAL;
  u->conv_path = path;
  return REG_OK;
}

const char* reg_unet_last_error(const reg_unet* u) { return u ? u->err.c_str() : "null network"; }

}  // extern "C"
