// Device building blocks of the semi-Lagrangian kernels, shared by the
// per-step kernels (transport.cu) and the persistent matvec kernel
// (matvec.cu): the periodic cubic B-spline prefilter on a 32x32 tile and the
// 4x4 periodic cubic interpolation stencil (§3.2, §3.5 "Interpolation").
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace regnk {

// Grid index helpers. P2 = true when both grid lengths are powers of two:
// indices split and wrap with shifts and masks (log1 = log2(n1)); otherwise
// (lengths 3 * 2^k) with integer division and remainder. The kernels are
// compiled for both, so the power-of-two grids pay nothing for the others.
template <bool P2>
__device__ __forceinline__ void split_index(long long idx, int n1, int log1, int& i, int& j) {
  if (P2) {
    i = (int)(idx & (n1 - 1));
    j = (int)(idx >> log1);
  } else {
    j = (int)(idx / n1);
    i = (int)(idx - (long long)j * n1);
  }
}

template <bool P2>
__device__ __forceinline__ long long row_offset(int j, int n1, int log1) {
  return P2 ? ((long long)j << log1) : (long long)j * n1;
}

// periodic wrap of any index into [0, n)
template <bool P2>
__device__ __forceinline__ int wrap_index(int i, int n) {
  if (P2) return i & (n - 1);
  const int r = i % n;
  return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// Periodic cubic B-spline prefilter.
//
// The spline interpolant sum_m c[m] beta3(x - m) takes the node values
// (c[k-1] + 4 c[k] + c[k+1]) / 6 per axis, so the coefficients are the
// samples filtered by the inverse of that symbol. The inverse factors into a
// causal and an anticausal first-order recursion with pole z1 = sqrt(3) - 2:
//     y[k] = s[k] + z1 y[k-1],   c'[k] = y[k] + z1 c'[k+1],   c = -6 z1 c'.
// A block filters a 32x32 output tile: it stages the tile with a periodic
// halo of kL = 12 samples on every side in shared memory. Along x, each of
// 4 threads per staged row produces 8 consecutive outputs, starting both
// recursions kL samples outside its segment (the truncated start-up terms
// decay as |z1|^12 < 1.5e-7, the order of the FP32 rounding of the
// recursions themselves); along y, 4 threads per column do the same. About
// 7 FMAs per sample and pass, in dependency chains of 52 steps with 224 (x)
// and 128 (y) threads of the block busy. kL is a multiple of 4 so that the
// staged region of a fused step kernel's box (which starts kL + 8 or kL + 16
// samples left of a tile) begins on a 16-byte boundary: its rows are staged
// with aligned float4 stores, and each chain of 32 samples is 8 float4.
constexpr float kZ1 = -0.26794919243112270f;    // sqrt(3) - 2
constexpr float kGain = 1.60769515458673624f;   // -6 z1
constexpr int kL = 12;              // recursion start-up length (halo width)
constexpr int kPX = 32, kPY = 32;   // output tile
constexpr int kPW = kPX + 2 * kL;   // staged tile width  (56)
constexpr int kPH = kPY + 2 * kL;   // staged tile height (56)
constexpr int kPIn = kPW + 1;       // odd pitches: conflict-free row and column walks
constexpr int kPMid = kPX + 1;
constexpr int kPThreads = 256;

// both recursions over n staged samples v[0..n-1]; outputs for k in
// [kL, kL + m) are written through out(k - kL, value)
template <int NS, int M, typename Out>
__device__ __forceinline__ void bspline_recursions(float (&v)[NS], Out out) {
#pragma unroll
  for (int k = 1; k < NS; ++k) v[k] = fmaf(kZ1, v[k - 1], v[k]);
  float c = v[NS - 1];
#pragma unroll
  for (int k = NS - 2; k >= kL; --k) {
    c = fmaf(kZ1, c, v[k]);
    if (k < kL + M) out(k - kL, kGain * c);
  }
}

// Prefilters the 32x32 output tile at (x0, y0) of one field (all kPThreads
// threads of the block take part; `sin_` and `smid` are the block's staging
// buffers of kPH*kPIn and kPH*kPMid floats). COHERENT = true reads the source
// with ordinary (L1-cached, non read-only-path) loads, for data written
// earlier in the same kernel by other blocks: the grid barrier's fences make
// such loads observe those writes, which the read-only path does not
// promise. The caller synchronises before reusing the buffers.
template <bool P2, bool COHERENT = false>
__device__ __forceinline__ void prefilter_tile(const float* __restrict__ src, float* __restrict__ dst,
                                               int n1, int n2, int log1, int x0, int y0,
                                               float* sin_, float* smid) {
  const int t = threadIdx.x;
  // all loads of the staged tile are issued before any shared-memory store,
  // so their latencies overlap
  constexpr int kLoads = (kPH * kPW + kPThreads - 1) / kPThreads;
  float ld_[kLoads];
#pragma unroll
  for (int u = 0; u < kLoads; ++u) {
    const int q = t + u * kPThreads;
    if (q < kPH * kPW) {
      const int r = q / kPW, c = q - r * kPW;
      const int gx = P2 ? wrap_index<true>(x0 - kL + c, n1) : wrap_once(x0 - kL + c, n1);
      const int gy = P2 ? wrap_index<true>(y0 - kL + r, n2) : wrap_once(y0 - kL + r, n2);
      const float* a = src + row_offset<P2>(gy, n1, log1) + gx;
      ld_[u] = COHERENT ? __ldca(a) : __ldg(a);
    }
  }
#pragma unroll
  for (int u = 0; u < kLoads; ++u) {
    const int q = t + u * kPThreads;
    if (q < kPH * kPW) {
      const int r = q / kPW, c = q - r * kPW;
      sin_[r * kPIn + c] = ld_[u];
    }
  }
  __syncthreads();
  constexpr int kSeg = 8, kSegs = kPX / kSeg, kLen = kSeg + 2 * kL;   // 32 samples per chain
  if (t < kPH * kSegs) {   // x recursions: staged row t % kPH, segment t / kPH
    // (a warp walks 32 consecutive rows of one segment: with the odd pitch
    // its shared-memory accesses fall in 32 different banks)
    const int r = t % kPH, sg = t / kPH;
    float v[kLen];
#pragma unroll
    for (int k = 0; k < kLen; ++k) v[k] = sin_[r * kPIn + sg * kSeg + k];
    float* row = smid + r * kPMid + sg * kSeg;
    bspline_recursions<kLen, kSeg>(v, [&](int o, float x) { row[o] = x; });
  }
  __syncthreads();
  if (t < kPX * kSegs) {   // y recursions: column t % 32, segment t / 32
    const int c = t % kPX, sg = t / kPX;
    float v[kLen];
#pragma unroll
    for (int k = 0; k < kLen; ++k) v[k] = smid[(sg * kSeg + k) * kPMid + c];
    float* col = dst + x0 + c;
    const int yb = y0 + sg * kSeg;
    bspline_recursions<kLen, kSeg>(v, [&](int o, float x) {
      col[row_offset<P2>(yb + o, n1, log1)] = x;
    });
  }
}

// Spline coefficients of one field on the W x W box of nodes whose first
// node is (bx0, by0) (periodic), left in shared memory for a gather that
// follows in the same block: box[r * (W + 1) + c] is the coefficient of node
// (bx0 + c, by0 + r); all NT threads of the block take part. The box's
// samples with a kL-sample halo are staged in
// `stage` (W + 2 kL rows of pitch PS) and the x pass goes to `mid`
// (transposed: W rows of pitch PT); `box` may alias `stage`. Same
// recursions and segment length as prefilter_tile, so the coefficients are
// those of k_prefilter up to the order of FP32 rounding. Ends with a block
// barrier.
// Pitches of the staged samples (rows) and of the x-pass output (stored
// transposed, one column of the box per row of `mid`): multiples of 4 floats
// with an odd quotient, so that each recursion chain reads its 32
// consecutive samples as float4 and the 8 chains of a quarter warp (8
// consecutive rows or columns) hit 8 different 16-byte bank groups.
constexpr int quad_pitch(int n) { return ((n + 3) / 4) % 2 ? (n + 3) / 4 * 4 : (n + 3) / 4 * 4 + 4; }

template <int W>
struct BoxDims {
  static constexpr int WS = W + 2 * kL;      // staged width and height
  static constexpr int PS = quad_pitch(WS);  // row pitch of the staged samples
  static constexpr int PT = quad_pitch(WS);  // row pitch of the transposed x-pass output
  // pitch of the coefficient box, 16 mod 32: the two tile rows a warp
  // gathers for (16 lanes each) fall in opposite halves of the banks
  static constexpr int PB = W + (48 - W % 32) % 32;
  static constexpr int kStage = WS * PS;     // floats
  static constexpr int kMid = W * PT;
  static constexpr size_t kSmemBytes = sizeof(float) * (kStage + kMid);
  static_assert(PS >= WS + 2 && PT >= WS + 2, "float4 reads run 2 samples past a chain");
  static_assert(PB % 32 == 16 && W * PB <= kStage, "the box fits the staging buffer it reuses");
};

// float4 vectors per staged row (the first one starts at the 4-aligned
// column at or left of the staged region's first column)
template <int W>
constexpr int box_row_vectors() { return (BoxDims<W>::WS + 3 + 3) / 4; }

// Places the float4 vector v = (e0..e3) of staged row r (first column `off`
// left of the staged region) into the staging buffer.
template <int W>
__device__ __forceinline__ void put_staged(float* stage, int r, int v, int off, float4 x) {
  using D = BoxDims<W>;
  if (off == 0 && 4 * v + 3 < D::WS) {   // aligned whole vector (PS % 4 == 0)
    *reinterpret_cast<float4*>(stage + r * D::PS + 4 * v) = x;
    return;
  }
  const float e[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = 4 * v + k - off;
    if (c >= 0 && c < D::WS) stage[r * D::PS + c] = e[k];
  }
}

// Outputs per recursion chain of the box prefilter (a chain reads kL
// samples more on each side). 8 gives the segments of k_prefilter (the same
// coefficients to the bit).
constexpr int kBoxSeg = 8;

// The two recursion passes of prefilter_box on samples already staged
// (stage[r * PS + c] = sample at node (bx0 - kL + c, by0 - kL + r)); ends
// with a block barrier.
template <int W, int NT>
__device__ __forceinline__ void box_recursions(float* stage, float* mid, float* box) {
  using D = BoxDims<W>;
  constexpr int WS = D::WS, PS = D::PS, PT = D::PT, PB = D::PB;
  const int t = threadIdx.x;
  constexpr int kSeg = kBoxSeg, kSegs = W / kSeg, kLen = kSeg + 2 * kL;
  static_assert(W % kSeg == 0 && kSeg % 4 == 0, "whole float4-aligned segments");
  constexpr int kQ = (kLen + 3) / 4;   // float4 reads per chain
  // x recursions: a warp walks 32 consecutive staged rows of one segment;
  // the outputs go to mid transposed (mid[column * PT + row])
  for (int q = t; q < WS * kSegs; q += NT) {
    const int r = q % WS, sg = q / WS;
    float v[kQ * 4];
    const float4* src4 = reinterpret_cast<const float4*>(stage + r * PS + sg * kSeg);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float4 x = src4[i];
      v[4 * i] = x.x;
      v[4 * i + 1] = x.y;
      v[4 * i + 2] = x.z;
      v[4 * i + 3] = x.w;
    }
    float* col = mid + sg * kSeg * PT + r;
    bspline_recursions<kLen, kSeg>(reinterpret_cast<float(&)[kLen]>(v),
                                   [&](int o, float x) { col[o * PT] = x; });
  }
  __syncthreads();
  // y recursions: a warp walks 32 consecutive box columns of one segment,
  // each reading its column of the x-pass output as float4
  for (int q = t; q < W * kSegs; q += NT) {
    const int c = q % W, sg = q / W;
    float v[kQ * 4];
    const float4* src4 = reinterpret_cast<const float4*>(mid + c * PT + sg * kSeg);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float4 x = src4[i];
      v[4 * i] = x.x;
      v[4 * i + 1] = x.y;
      v[4 * i + 2] = x.z;
      v[4 * i + 3] = x.w;
    }
    float* colb = box + sg * kSeg * PB + c;
    bspline_recursions<kLen, kSeg>(reinterpret_cast<float(&)[kLen]>(v),
                                   [&](int o, float x) { colb[o * PB] = x; });
  }
  __syncthreads();
}

template <int W, bool P2, int NT = kPThreads>
__device__ __forceinline__ void prefilter_box(const float* __restrict__ src, int n1, int n2,
                                              int log1, int bx0, int by0, float* stage,
                                              float* mid, float* box) {
  using D = BoxDims<W>;
  constexpr int WS = D::WS;
  // The staged rows are read as float4 from a 4-aligned first column (a
  // float4 never straddles the periodic seam since n1 % 4 == 0) and the
  // first `off` columns of the first vector are dropped. Row-major thread
  // order keeps the loads of a warp contiguous.
  constexpr int kV = box_row_vectors<W>();      // float4 per staged row
  constexpr int kLoads = (WS * kV + NT - 1) / NT;
  const int cx0 = bx0 - kL;
  const int ax0 = cx0 & ~3;
  const int off = cx0 - ax0;
  const int t = threadIdx.x;
  float4 ld_[kLoads];
#pragma unroll
  for (int u = 0; u < kLoads; ++u) {
    const int q = t + u * NT;
    if (q < WS * kV) {
      const int r = q / kV, v = q - r * kV;
      const int gx = P2 ? wrap_index<true>(ax0 + 4 * v, n1) : wrap_once(ax0 + 4 * v, n1);
      const int gy = P2 ? wrap_index<true>(by0 - kL + r, n2) : wrap_once(by0 - kL + r, n2);
      ld_[u] = __ldg(reinterpret_cast<const float4*>(src + row_offset<P2>(gy, n1, log1) + gx));
    }
  }
#pragma unroll
  for (int u = 0; u < kLoads; ++u) {
    const int q = t + u * NT;
    if (q < WS * kV) {
      const int r = q / kV, v = q - r * kV;
      put_staged<W>(stage, r, v, off, ld_[u]);
    }
  }
  __syncthreads();
  box_recursions<W, NT>(stage, mid, box);
}

// ---------------------------------------------------------------------------
// 4x4 periodic cubic interpolation at node (i, j) + (d1, d2) cells.
struct Stencil {
  int ii[4];
  int jj[4];   // row offsets (already multiplied by n1)
  float w1[4], w2[4];
};

__device__ __forceinline__ void cubic_weights(float t, float (&w)[4], bool lagrange) {
  if (lagrange) {  // cubic Lagrange on nodes -1, 0, 1, 2
    const float tm1 = t - 1.f, tm2 = t - 2.f, tp1 = t + 1.f;
    w[0] = -t * tm1 * tm2 * (1.f / 6.f);
    w[1] = tp1 * tm1 * tm2 * 0.5f;
    w[2] = -tp1 * t * tm2 * 0.5f;
    w[3] = tp1 * t * tm1 * (1.f / 6.f);
  } else {         // centred cubic B-spline
    const float s = 1.f - t, t2 = t * t, t3 = t2 * t;
    w[0] = s * s * s * (1.f / 6.f);
    w[1] = (3.f * t3 - 6.f * t2 + 4.f) * (1.f / 6.f);
    w[2] = (-3.f * t3 + 3.f * t2 + 3.f * t + 1.f) * (1.f / 6.f);
    w[3] = t3 * (1.f / 6.f);
  }
}

template <bool P2>
__device__ __forceinline__ Stencil make_stencil(int i, int j, float d1, float d2, int n1,
                                                int n2, int log1, bool lagrange) {
  Stencil S;
  const float f1 = floorf(d1), f2 = floorf(d2);
  cubic_weights(d1 - f1, S.w1, lagrange);
  cubic_weights(d2 - f2, S.w2, lagrange);
  const int i0 = wrap_index<P2>(i + (int)f1 - 1, n1), j0 = wrap_index<P2>(j + (int)f2 - 1, n2);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int ii = i0 + a, jj = j0 + a;
    S.ii[a] = ii < n1 ? ii : ii - n1;
    S.jj[a] = (int)row_offset<P2>(jj < n2 ? jj : jj - n2, n1, log1);
  }
  return S;
}

// COHERENT: ordinary cached load (see prefilter_tile); otherwise read-only path
template <bool COHERENT = false>
__device__ __forceinline__ float ld(const float* p) { return COHERENT ? __ldca(p) : __ldg(p); }

template <bool COHERENT = false>
__device__ __forceinline__ float apply_stencil(const Stencil& S, const float* __restrict__ c) {
  float acc = 0.f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const float* row = c + S.jj[b];
    const float r = S.w1[0] * ld<COHERENT>(row + S.ii[0]) + S.w1[1] * ld<COHERENT>(row + S.ii[1]) +
                    S.w1[2] * ld<COHERENT>(row + S.ii[2]) + S.w1[3] * ld<COHERENT>(row + S.ii[3]);
    acc = fmaf(S.w2[b], r, acc);
  }
  return acc;
}

// The 4x4 sum of apply_stencil over coefficients held in a shared-memory box
// of pitch PB: node (i0 + a, j0 + b) of the stencil is box entry
// (li + a, lj + b). The caller clamps li, lj to [0, W - 4].
template <int PB>
__device__ __forceinline__ float apply_box(const float* box, int li, int lj, const float (&w1)[4],
                                           const float (&w2)[4]) {
  float acc = 0.f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const float* row = box + (lj + b) * PB + li;
    const float r = w1[0] * row[0] + w1[1] * row[1] + w1[2] * row[2] + w1[3] * row[3];
    acc = fmaf(w2[b], r, acc);
  }
  return acc;
}

}  // namespace regnk
