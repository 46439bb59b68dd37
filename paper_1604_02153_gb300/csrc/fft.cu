// Hand-written shared-memory 2D real FFT fused with the pointwise spectral
// multipliers of the pseudospectral discretisation (§3.2; eq. diffopregv;
// eq. reg-precond; §3.4.2 restriction, prolongation and cut-off filters).
//
// A spectral operator out = F^-1[ sigma(k) F[in] ] runs as three kernels:
//   1. rows_r2c : forward FFT along x_1 of every row. Two real rows are packed
//                 into one complex line (z = a + i b) and separated after the
//                 transform; the half spectrum k1 = 0..n1/2 is written line by
//                 line (one line per k1, contiguous over the rows j).
//   2. cols     : for each k1 line: forward FFT along x_2, multiply by
//                 sigma(k1, k2) (combining several inputs and producing several
//                 outputs where the operator needs it: grad, div), optional
//                 resampling to a grid of half or double size (spectral
//                 restriction / prolongation), inverse FFT along x_2.
//   3. rows_c2r : inverse FFT along x_1, two rows per complex line, with an
//                 optional addend fused into the store.
// Each transform is a Stockham autosort FFT in shared memory: radix-8
// passes (8-point DFTs in registers), one radix-4 or radix-2 pass for the
// rest of 2^L, and a radix-3 pass for lengths 3 * 2^L, with FP32 twiddles
// rounded from an FP64 host table. Normalisation (1/N of the input grid) is
// folded into sigma.
#include "common.cuh"
#include "kernels.h"

namespace regnk {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Line lengths N = 2^L * 3^T (T = 0 or 1). Lines per block and threads per
// block of the FFT kernels: P lines of N complex values, P a power of two
// with P N <= 2048 (at most 16 KB of shared memory per block) and P = 1
// from N = 512 on, so that a 512^2 grid gives 256 blocks per field and pass
// and 1024^2 over 500 (fewer, larger blocks measured slower at both sizes).
// Elements per thread in the load and store phases of the FFT kernels. The
// radix-8 passes have P N / 8 butterflies, so with 4 half of the threads wait
// during them; 8 (every thread busy, half the threads) measured slower
// (1024^2 operator 38.8 against 36.6 us: spills in the column pass).
constexpr int kFftPer = 4;

template <int L, int T>
struct FftCfg {
  static constexpr int N = (1 << L) * (T ? 3 : 1);
  static constexpr int P = N >= 512 ? 1 : (N >= 256 ? 4 : (N >= 128 ? 8 : 16));
  static constexpr int NT = (P * N / kFftPer) < 256 ? P * N / kFftPer : 256;
};

// Lines per block and threads of the row passes (k_rows_r2c, k_rows_c2r): P
// line pairs per block; each pass writes or reads 2 P adjacent values of
// every spectral line.
template <int L, int T>
struct RowCfg {
  static constexpr int N = FftCfg<L, T>::N;
  // two line pairs per block from N = 1024: each spectral line then receives
  // 32 contiguous bytes (a whole sector) per block (grad at 1024^2: 38 -> 34 us)
  static constexpr int P = N >= 1024 ? 2 : FftCfg<L, T>::P;
  static constexpr int NT = (P * N / kFftPer) < 256 ? P * N / kFftPer : 256;
};

// 8-point DFT in registers: two 4-point DFTs of the even and odd inputs,
// the odd ones turned by W8^s, then the radix-2 combination (forward
// W = exp(-2 pi i / 8), inverse its conjugate).
template <bool INV>
__device__ __forceinline__ void dft4(float2 a0, float2 a1, float2 a2, float2 a3, float2& y0,
                                     float2& y1, float2& y2, float2& y3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const float2 s13 = cadd(a1, a3), d13 = mul_mi<INV>(csub(a1, a3));
  y0 = cadd(s02, s13);
  y1 = cadd(d02, d13);
  y2 = csub(s02, s13);
  y3 = csub(d02, d13);
}

template <bool INV>
__device__ __forceinline__ void dft8(const float2 (&a)[8], float2 (&y)[8]) {
  constexpr float kR2 = 0.70710678118654752f;   // sqrt(2) / 2
  float2 e0, e1, e2, e3, o0, o1, o2, o3;
  dft4<INV>(a[0], a[2], a[4], a[6], e0, e1, e2, e3);
  dft4<INV>(a[1], a[3], a[5], a[7], o0, o1, o2, o3);
  // o_s *= W8^s
  o1 = INV ? make_float2(kR2 * (o1.x - o1.y), kR2 * (o1.x + o1.y))
           : make_float2(kR2 * (o1.x + o1.y), kR2 * (o1.y - o1.x));
  o2 = mul_mi<INV>(o2);
  o3 = INV ? make_float2(-kR2 * (o3.x + o3.y), kR2 * (o3.x - o3.y))
           : make_float2(kR2 * (o3.y - o3.x), -kR2 * (o3.x + o3.y));
  y[0] = cadd(e0, o0); y[4] = csub(e0, o0);
  y[1] = cadd(e1, o1); y[5] = csub(e1, o1);
  y[2] = cadd(e2, o2); y[6] = csub(e2, o2);
  y[3] = cadd(e3, o3); y[7] = csub(e3, o3);
}

// Shared-memory position of element i of a block's FFT buffer: the low four
// bits of i are XORed with bits 3..6 (a permutation inside each aligned run
// of 16 float2). The Stockham passes store with strides 8 and 64 (radix-8
// passes one and two), which put 8 or 4 lanes of a half-warp on the same
// bank; with this permutation every pass and every aligned contiguous run is
// conflict-free. Buffers start on multiples of 128 elements, so a buffer's
// permutation does not depend on where it sits in shared memory.
__device__ __forceinline__ int sw(int i) { return i ^ ((i >> 3) & 15); }

// In-place FFT of P lines of length N = 2^L 3^T stored contiguously at s
// (line l at s + l*N): radix-8 Stockham passes, then one radix-4 or radix-2
// pass for the remaining factor of 2^L, then a radix-3 pass if T = 1, each
// pass reading its inputs into registers, synchronising and writing its
// outputs. All NT threads of the block take part; the caller synchronises
// before (data written) and the routine ends with a barrier. tw holds
// exp(-2 pi i m / N), m < N.
template <int L, int T, int P, int NT, bool INV>
__device__ void fft_smem(float2* s, const float2* __restrict__ tw) {
  constexpr int N = (1 << L) * (T ? 3 : 1);
  const int t = threadIdx.x;
  int lns = 0;  // log2 of the current sub-transform size Ns
  constexpr int Q8 = N / 8;
  constexpr int TOT8 = P * Q8;
  constexpr int B8 = (TOT8 + NT - 1) / NT;
#pragma unroll   // constant twiddle strides per pass
  for (int pass = 0; pass < L / 3; ++pass) {
    const int Ns = 1 << lns;
    const int tws = N >> (lns + 3);  // twiddle stride N / (8 Ns)
    float2 v[B8][8];
    int base[B8];
#pragma unroll
    for (int b = 0; b < B8; ++b) {
      const int q = t + b * NT;
      if (TOT8 % NT == 0 || q < TOT8) {
        const int l = q / Q8, j = q % Q8;
        const int k = j & (Ns - 1);
        float2 a[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) a[r] = s[sw(l * N + j + r * Q8)];
        if (lns > 0) {
#pragma unroll
          for (int r = 1; r < 8; ++r) {
            const float2 w = __ldg(tw + r * k * tws);
            a[r] = INV ? cmulc(a[r], w) : cmul(a[r], w);
          }
        }
        dft8<INV>(a, v[b]);
        base[b] = l * N + (j - k) * 8 + k;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B8; ++b) {
      const int q = t + b * NT;
      if (TOT8 % NT == 0 || q < TOT8) {
#pragma unroll
        for (int r = 0; r < 8; ++r) s[sw(base[b] + r * Ns)] = v[b][r];
      }
    }
    __syncthreads();
    lns += 3;
  }
  if (L % 3 == 2) {
    constexpr int Q4 = N / 4;
    constexpr int TOT4 = P * Q4;
    constexpr int B4 = (TOT4 + NT - 1) / NT;
    const int Ns = 1 << lns;
    const int tws = N >> (lns + 2);  // twiddle stride N / (4 Ns)
    float2 v[B4][4];
    int base[B4];
#pragma unroll
    for (int b = 0; b < B4; ++b) {
      const int q = t + b * NT;
      if (TOT4 % NT == 0 || q < TOT4) {
        const int l = q / Q4, j = q % Q4;
        const int k = j & (Ns - 1);
        const int x = l * N + j;
        float2 a0 = s[sw(x)], a1 = s[sw(x + Q4)], a2 = s[sw(x + 2 * Q4)], a3 = s[sw(x + 3 * Q4)];
        if (lns > 0) {
          const float2 w1 = __ldg(tw + k * tws);
          const float2 w2 = __ldg(tw + 2 * k * tws);
          const float2 w3 = __ldg(tw + 3 * k * tws);
          if (INV) {
            a1 = cmulc(a1, w1); a2 = cmulc(a2, w2); a3 = cmulc(a3, w3);
          } else {
            a1 = cmul(a1, w1); a2 = cmul(a2, w2); a3 = cmul(a3, w3);
          }
        }
        dft4<INV>(a0, a1, a2, a3, v[b][0], v[b][1], v[b][2], v[b][3]);
        base[b] = l * N + (j - k) * 4 + k;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B4; ++b) {
      const int q = t + b * NT;
      if (TOT4 % NT == 0 || q < TOT4) {
        s[sw(base[b])] = v[b][0];
        s[sw(base[b] + Ns)] = v[b][1];
        s[sw(base[b] + 2 * Ns)] = v[b][2];
        s[sw(base[b] + 3 * Ns)] = v[b][3];
      }
    }
    __syncthreads();
    lns += 2;
  }
  if (L % 3 == 1) {
    constexpr int Q2 = N / 2;
    constexpr int TOT2 = P * Q2;
    constexpr int B2 = (TOT2 + NT - 1) / NT;
    const int Ns = 1 << lns;
    const int tws = N >> (lns + 1);  // N / (2 Ns)
    float2 v0[B2], v1[B2];
    int base[B2];
#pragma unroll
    for (int b = 0; b < B2; ++b) {
      const int q = t + b * NT;
      if (TOT2 % NT == 0 || q < TOT2) {
        const int l = q / Q2, j = q % Q2;
        const int k = j & (Ns - 1);
        const float2 a0 = s[sw(l * N + j)];
        float2 a1 = s[sw(l * N + j + Q2)];
        if (lns > 0) {
          const float2 w = __ldg(tw + k * tws);
          a1 = INV ? cmulc(a1, w) : cmul(a1, w);
        }
        v0[b] = cadd(a0, a1);
        v1[b] = csub(a0, a1);
        base[b] = l * N + (j - k) * 2 + k;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B2; ++b) {
      const int q = t + b * NT;
      if (TOT2 % NT == 0 || q < TOT2) {
        s[sw(base[b])] = v0[b];
        s[sw(base[b] + Ns)] = v1[b];
      }
    }
    __syncthreads();
    lns += 1;
  }
  if (T) {
    // radix 3 with Ns = 2^L = N / 3: k = j, output at k + s Ns
    constexpr int Q3 = N / 3;
    constexpr int TOT3 = P * Q3;
    constexpr int B3 = (TOT3 + NT - 1) / NT;
    constexpr float kS3 = 0.86602540378443865f;   // sqrt(3) / 2
    float2 v0[B3], v1[B3], v2[B3];
    int base[B3];
#pragma unroll
    for (int b = 0; b < B3; ++b) {
      const int q = t + b * NT;
      if (TOT3 % NT == 0 || q < TOT3) {
        const int l = q / Q3, k = q % Q3;
        const float2 a0 = s[sw(l * N + k)];
        float2 a1 = s[sw(l * N + k + Q3)], a2 = s[sw(l * N + k + 2 * Q3)];
        if (L > 0) {
          const float2 w1 = __ldg(tw + k), w2 = __ldg(tw + 2 * k);
          a1 = INV ? cmulc(a1, w1) : cmul(a1, w1);
          a2 = INV ? cmulc(a2, w2) : cmul(a2, w2);
        }
        const float2 t1 = cadd(a1, a2), t2 = csub(a1, a2);
        const float2 m = make_float2(a0.x - 0.5f * t1.x, a0.y - 0.5f * t1.y);
        // forward: b1 = m - i (sqrt3/2) t2, b2 = m + i (sqrt3/2) t2
        const float2 it2 = INV ? make_float2(-kS3 * t2.y, kS3 * t2.x)
                               : make_float2(kS3 * t2.y, -kS3 * t2.x);
        v0[b] = cadd(a0, t1);
        v1[b] = cadd(m, it2);
        v2[b] = csub(m, it2);
        base[b] = l * N + k;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B3; ++b) {
      const int q = t + b * NT;
      if (TOT3 % NT == 0 || q < TOT3) {
        s[sw(base[b])] = v0[b];
        s[sw(base[b] + Q3)] = v1[b];
        s[sw(base[b] + 2 * Q3)] = v2[b];
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ bool field_skipped(const FieldMask& fm) {
  return fm.mask && !fm.mask[fm.p0 + (int)blockIdx.y / fm.per];
}

// ---------------------------------------------------------------------------
// 1. forward row transforms: F fields of n2 rows of length N = n1.
template <int L, int T>
__global__ void __launch_bounds__(RowCfg<L, T>::NT)
k_rows_r2c(const float* __restrict__ in, long long fstride, float2* __restrict__ spec,
           long long sstride, int n2, const float2* __restrict__ tw, FieldMask fm) {
  pdl_enter();
  if (field_skipped(fm)) return;
  constexpr int N = RowCfg<L, T>::N, P = RowCfg<L, T>::P, NT = RowCfg<L, T>::NT;
  extern __shared__ float2 sm[];
  const int t = threadIdx.x;
  const int row0 = blockIdx.x * 2 * P;
  const float* src = in + (long long)blockIdx.y * fstride;
  constexpr int LD = (P * N + NT - 1) / NT;   // loads issued before the stores
  float2 v[LD];
#pragma unroll
  for (int u = 0; u < LD; ++u) {
    const int q = t + u * NT;
    if ((P * N) % NT == 0 || q < P * N) {
      const int l = q / N, i = q % N;
      const long long r = (long long)(row0 + 2 * l) * N + i;
      v[u] = make_float2(__ldg(src + r), __ldg(src + r + N));
    }
  }
#pragma unroll
  for (int u = 0; u < LD; ++u) {
    const int q = t + u * NT;
    if ((P * N) % NT == 0 || q < P * N) sm[sw(q)] = v[u];
  }
  __syncthreads();
  fft_smem<L, T, P, NT, false>(sm, tw);
  float2* dst = spec + (long long)blockIdx.y * sstride;
  constexpr int R = 2 * P;
  for (int q = t; q < (N / 2 + 1) * R; q += NT) {
    const int r = q % R, k = q / R, l = r >> 1;
    const float2 Z = sm[sw(l * N + k)];
    const float2 Zm = sm[sw(l * N + (k == 0 ? 0 : N - k))];
    float2 X;
    if (r & 1) {  // X_b = (Z - conj(Zm)) / (2i)
      X = make_float2(0.5f * (Z.y + Zm.y), -0.5f * (Z.x - Zm.x));
    } else {      // X_a = (Z + conj(Zm)) / 2
      X = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
    }
    dst[(long long)k * n2 + row0 + r] = X;
  }
}

// 3. inverse row transforms (half spectrum -> real rows), optional addend.
// CHEB: the Chebyshev epilogue (a separate instantiation: its prefetched
// operands would otherwise set the register count of every inverse pass).
template <int L, int T, bool CHEB>
__global__ void __launch_bounds__(RowCfg<L, T>::NT)
k_rows_c2r(const float2* __restrict__ spec, long long sstride, float* __restrict__ out,
           long long fstride, const float* __restrict__ add, long long astride, int n2,
           const float2* __restrict__ tw, ChebEpilogue cheb, FieldMask fm) {
  pdl_enter();
  if (field_skipped(fm)) return;
  constexpr int N = RowCfg<L, T>::N, P = RowCfg<L, T>::P, NT = RowCfg<L, T>::NT;
  extern __shared__ float2 sm[];
  const int t = threadIdx.x;
  const int row0 = blockIdx.x * 2 * P;
  const float2* src = spec + (long long)blockIdx.y * sstride;
  // The epilogue's operands at this thread's output points (the addend, or
  // the Chebyshev vectors) are loaded first, so their latency overlaps the
  // transform
  constexpr int kOut = (P * N + NT - 1) / NT;
  float cr_[kOut][2], cd_[kOut][2], cx_[kOut][2];
  if (!CHEB && add) {   // plain pass: the addend is prefetched into cr_
    const float* ad0 = add + (long long)blockIdx.y * astride;
#pragma unroll
    for (int u = 0; u < kOut; ++u) {
      const int q = t + u * NT;
      if ((P * N) % NT == 0 || q < P * N) {
        const int l = q / N, i = q % N;
        const long long r = (long long)(row0 + 2 * l) * N + i;
        cr_[u][0] = __ldg(ad0 + r);
        cr_[u][1] = __ldg(ad0 + r + N);
      }
    }
  }
  if (CHEB) {
    const long long fo = (long long)blockIdx.y * fstride;
#pragma unroll
    for (int u = 0; u < kOut; ++u) {
      const int q = t + u * NT;
      if ((P * N) % NT == 0 || q < P * N) {
        const int l = q / N, i = q % N;
        const long long r = fo + (long long)(row0 + 2 * l) * N + i;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          cr_[u][h] = cheb.r[r + h * N];
          cd_[u][h] = cheb.d[r + h * N];
          cx_[u][h] = cheb.x[r + h * N];
        }
      }
    }
  }
  constexpr int TOT = (N / 2 + 1) * P;
  constexpr int LD = (TOT + NT - 1) / NT;     // loads issued before the stores
  float4 v[LD];
#pragma unroll
  for (int u = 0; u < LD; ++u) {
    const int q = t + u * NT;
    if (q < TOT) {
      const int l = q % P, k = q / P;
      const long long a = (long long)k * n2 + row0 + 2 * l;
      v[u] = __ldg(reinterpret_cast<const float4*>(src + a));   // X_a, X_b adjacent
    }
  }
#pragma unroll
  for (int u = 0; u < LD; ++u) {
    const int q = t + u * NT;
    if (q < TOT) {
      const int l = q % P, k = q / P;
      float2 Xa = make_float2(v[u].x, v[u].y), Xb = make_float2(v[u].z, v[u].w);
      if (k == 0 || k == N / 2) {
        Xa.y = 0.f;
        Xb.y = 0.f;
      }
      sm[sw(l * N + k)] = make_float2(Xa.x - Xb.y, Xa.y + Xb.x);
      if (k > 0 && k < N / 2) sm[sw(l * N + N - k)] = make_float2(Xa.x + Xb.y, Xb.x - Xa.y);
    }
  }
  __syncthreads();
  fft_smem<L, T, P, NT, true>(sm, tw);
  float* dst = out + (long long)blockIdx.y * fstride;
  const float* ad = add ? add + (long long)blockIdx.y * astride : nullptr;
  if (CHEB) {
    // Ad is never stored. The addend is d itself (already in cd_), and r, d
    // and x are read and overwritten here by the same thread.
    const long long fo = (long long)blockIdx.y * fstride;
    float* cr = cheb.r + fo;
    float* cd = cheb.d + fo;
    float* cx = cheb.x + fo;
#pragma unroll
    for (int u = 0; u < kOut; ++u) {
      const int q = t + u * NT;
      if ((P * N) % NT == 0 || q < P * N) {
        const int l = q / N, i = q % N;
        const long long r = (long long)(row0 + 2 * l) * N + i;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const long long e = r + h * N;
          const float2 o = sm[sw(q)];
          const float Ad = (h ? o.y : o.x) + (ad ? cd_[u][h] : 0.f);
          const float ri = cr_[u][h] - Ad;
          const float di = fmaf(cheb.a, cd_[u][h], cheb.b * ri);
          cr[e] = ri;
          cd[e] = di;
          cx[e] = cx_[u][h] + di;
        }
      }
    }
    return;
  }
#pragma unroll
  for (int u = 0; u < kOut; ++u) {
    const int q = t + u * NT;
    if ((P * N) % NT == 0 || q < P * N) {
      const int l = q / N, i = q % N;
      const long long r = (long long)(row0 + 2 * l) * N + i;
      const float2 o = sm[sw(q)];
      float a = o.x, b = o.y;
      if (ad) {
        a += cr_[u][0];
        b += cr_[u][1];
      }
      dst[r] = a;
      dst[r + N] = b;
    }
  }
}

// ---------------------------------------------------------------------------
// 2. column pass with the spectral multiplier.
__device__ __forceinline__ float regpow(float beta, int p, float s, int k1, int k2) {
  const float k2n = (float)k1 * (float)k1 + (float)k2 * (float)k2;
  float g = k2n;
  if (p == 2) g = k2n * k2n;
  else if (p == 3) g = k2n * k2n * k2n;
  if (s == 1.f) return beta * g;
  if (g == 0.f) g = 1.f;
  const float bg = beta * g;
  if (s == -1.f) return 1.f / bg;
  if (s == -0.5f) return 1.f / sqrtf(bg);
  if (s == 0.5f) return sqrtf(bg);
  return powf(bg, s);
}

// Leray projection K = I - grad (div grad)^-1 div (§3.1, the K of the
// gradient for an incompressible velocity): entry (o, c) of its symbol
// delta_oc - k_o k_c / |k|^2 with the derivative wavenumbers of grad and div
// (Nyquist zeroed), so that div K b vanishes for the discrete div; the
// identity on the modes where div grad vanishes.
__device__ __forceinline__ float leray(int o, int c, float kd1, float kd2) {
  const float q = kd1 * kd1 + kd2 * kd2;
  const float d = (o == c) ? 1.f : 0.f;
  if (q == 0.f) return d;
  return d - (o == 0 ? kd1 : kd2) * (c == 0 ? kd1 : kd2) / q;
}

// (beta g)^s for the powers the solver uses (s = 1, -1, -1/2, 1/2), powf
// otherwise
__device__ __forceinline__ float pow_s(float x, float s) {
  if (s == 1.f) return x;
  if (s == -1.f) return 1.f / x;
  if (s == -0.5f) return 1.f / sqrtf(x);
  if (s == 0.5f) return sqrtf(x);
  return powf(x, s);
}

// Entry (o, c) of R^s for the near-incompressible regularisation operator
// R = beta A - beta_w grad (I - Lap) div (§2: the H1 norm of the mass
// source w = div v, eq. varopt:regw, with w and p eliminated from the
// control equations eq. control-v and eq. control-w of Appendix A). Per
// wavenumber R is the symmetric 2 x 2 matrix a I + cw kd kd^T with
// a = beta |k|^2p (k = 0 weight 1 unless s = 1), cw = beta_w (1 + |k|^2) and
// kd the derivative wavenumbers (Nyquist zeroed): eigenvalue a + cw |kd|^2
// along kd, a across it, so
//     R^s = a^s I + ((a + cw |kd|^2)^s - a^s) kd kd^T / |kd|^2.
// (out of line, like kw below: inlined into the shared column-pass code they
// raised its register count for every operator)
__device__ __noinline__ float regw(float beta, int p, float s, float beta_w, int o, int c, int k1,
                                   int k2, float kd1, float kd2) {
  const float k2n = (float)k1 * (float)k1 + (float)k2 * (float)k2;
  float g = k2n;
  if (p == 2) g = k2n * k2n;
  else if (p == 3) g = k2n * k2n * k2n;
  const float d = (o == c) ? 1.f : 0.f;
  const float ko = o == 0 ? kd1 : kd2, kc = c == 0 ? kd1 : kd2;
  const float cw = beta_w * (1.f + k2n);
  if (s == 1.f) return beta * g * d + cw * ko * kc;
  if (g == 0.f) g = 1.f;
  const float av = beta * g;
  const float q = kd1 * kd1 + kd2 * kd2;
  const float as = pow_s(av, s);
  if (q == 0.f) return as * d;
  return as * d + (pow_s(av + cw * q, s) - as) * ko * kc / q;
}

// Entry (o, c) of the near-incompressible K of the reduced gradient and the
// Hessian (eq. control-elim, eq. hessian-matvec). Eliminating w and p from
// the control equations gives beta A v - beta_w grad (I - Lap) div v + b = 0,
// i.e. beta A v + K[b] = 0 with K = beta A M^-1, M = beta A - beta_w grad
// (I - Lap) div; per wavenumber M = a I + cw kd kd^T (see regw), so
//     K = I - c kd kd^T / |kd|^2,  c = cw |kd|^2 / (a + cw |kd|^2)  in [0, 1)
// (the identity where kd = 0; c -> 1 is the Leray projection, c -> 0 the
// identity). Its symbol is bounded, unlike M's.
__device__ __noinline__ float kw(float beta, int p, float beta_w, int o, int c, int k1, int k2,
                                 float kd1, float kd2) {
  const float q = kd1 * kd1 + kd2 * kd2;
  const float d = (o == c) ? 1.f : 0.f;
  if (q == 0.f) return d;
  const float k2n = (float)k1 * (float)k1 + (float)k2 * (float)k2;
  float g = k2n;
  if (p == 2) g = k2n * k2n;
  else if (p == 3) g = k2n * k2n * k2n;
  const float cq = beta_w * (1.f + k2n) * q;
  const float w = cq / (beta * g + cq);
  return d - w * (o == 0 ? kd1 : kd2) * (c == 0 ? kd1 : kd2) / q;
}

// sigma_{o,c}(k1, k2) as a complex number; k1 >= 0, k2 signed; n1, n2 of the
// grid the Nyquist and filter conditions refer to.
__device__ __forceinline__ float2 symbol(const ColArgs& a, int o, int c, int k1, int k2) {
  const bool nyq1 = (k1 == a.n1 / 2), nyq2 = (k2 == -a.n2 / 2);
  const bool low = (k1 < a.n1 / 4) && (k2 < a.n2 / 4) && (k2 > -a.n2 / 4);
  switch (a.op) {
    case SPOP_SCALE:
      return make_float2(1.f, 0.f);
    case SPOP_GRAD:
      if (o == 0) return make_float2(0.f, nyq1 ? 0.f : (float)k1);
      return make_float2(0.f, nyq2 ? 0.f : (float)k2);
    case SPOP_DIV:
      if (c == 0) return make_float2(0.f, nyq1 ? 0.f : (float)k1);
      return make_float2(0.f, nyq2 ? 0.f : (float)k2);
    case SPOP_REGPOW:
      return make_float2(regpow(a.beta, a.p, a.s, k1, k2), 0.f);
    case SPOP_LOWPASS:
      return make_float2(low ? 1.f : 0.f, 0.f);
    case SPOP_HIGHPASS:
      return make_float2(low ? 0.f : 1.f, 0.f);
    case SPOP_REGPOW_HIGH:
      return make_float2(low ? 0.f : regpow(a.beta, a.p, a.s, k1, k2), 0.f);
    case SPOP_LERAY:
      return make_float2(leray(o, c, nyq1 ? 0.f : (float)k1, nyq2 ? 0.f : (float)k2), 0.f);
    case SPOP_REGPOW_LERAY:
      return make_float2(regpow(a.beta, a.p, a.s, k1, k2) *
                             leray(o, c, nyq1 ? 0.f : (float)k1, nyq2 ? 0.f : (float)k2),
                         0.f);
    case SPOP_REGW:
      return make_float2(regw(a.beta, a.p, a.s, a.beta_w, o, c, k1, k2, nyq1 ? 0.f : (float)k1,
                              nyq2 ? 0.f : (float)k2),
                         0.f);
    case SPOP_KW:
      return make_float2(kw(a.beta, a.p, a.beta_w, o, c, k1, k2, nyq1 ? 0.f : (float)k1,
                            nyq2 ? 0.f : (float)k2),
                         0.f);
    case SPOP_REGPOW_KW:
      return make_float2(regpow(a.beta, a.p, a.s, k1, k2) *
                             kw(a.beta, a.p, a.beta_w, o, c, k1, k2, nyq1 ? 0.f : (float)k1,
                                nyq2 ? 0.f : (float)k2),
                         0.f);
    default:
      return make_float2(0.f, 0.f);
  }
}

// Column pass between input lines of 2^LI 3^T and output lines of 2^LO 3^T.
template <int LI, int LO, int T>
struct ColCfg {
  static constexpr int LM = LI > LO ? LI : LO;
  static constexpr int NM = FftCfg<LM, T>::N;
  static constexpr int P = FftCfg<LM, T>::P;
  static constexpr int NT = FftCfg<LM, T>::NT;
};

// 64 registers per thread at most (1024 threads' worth of blocks per SM):
// left to itself the compiler gave the 1024-point column pass 108 registers,
// two blocks per SM
template <int LI, int LO, int T>
__global__ void __launch_bounds__(ColCfg<LI, LO, T>::NT, 1024 / ColCfg<LI, LO, T>::NT) k_cols(ColArgs a) {
  pdl_enter();
  if (field_skipped(a.fm)) return;
  constexpr int NI = FftCfg<LI, T>::N, NO = FftCfg<LO, T>::N;
  constexpr int NM = ColCfg<LI, LO, T>::NM;
  constexpr int P = ColCfg<LI, LO, T>::P, NT = ColCfg<LI, LO, T>::NT;
  extern __shared__ float2 sm[];
  float2* bin = sm;                      // nin buffers of P x NM
  float2* bout = sm + a.nin * P * NM;    // 1 buffer of P x NM
  const int t = threadIdx.x;
  const int line0 = blockIdx.x * P;
  const int g = blockIdx.y;
  const int nsmall = a.n1_in < a.n1_out ? a.n1_in : a.n1_out;
  const bool resize = (NI != NO) || (a.n1_in != a.n1_out);
  constexpr int LD = (P * NI + NT - 1) / NT;   // loads issued before the stores
  for (int c = 0; c < a.nin; ++c) {
    const float2* src = a.in + (long long)(g * a.nin + c) * a.in_fstride;
    float2 v[LD];
#pragma unroll
    for (int u = 0; u < LD; ++u) {
      const int q = t + u * NT;
      v[u] = make_float2(0.f, 0.f);
      if (q < P * NI) {
        const int l = q / NI, k2 = q % NI;
        const int k1 = line0 + l;
        const bool ok = k1 < a.nk1_out && (!resize || k1 < nsmall / 2);
        if (ok) v[u] = __ldg(src + (long long)k1 * NI + k2);
      }
    }
#pragma unroll
    for (int u = 0; u < LD; ++u) {
      const int q = t + u * NT;
      if (q < P * NI) bin[c * P * NM + sw(q)] = v[u];
    }
  }
  __syncthreads();
  for (int c = 0; c < a.nin; ++c) fft_smem<LI, T, P, NT, false>(bin + c * P * NM, a.tw_in);
  for (int o = 0; o < a.nout; ++o) {
    for (int q = t; q < P * NO; q += NT) {
      const int l = q / NO, ko = q % NO;
      const int k1 = line0 + l;
      const int k2 = signed_k(ko, NO);
      bool ok = k1 < a.nk1_out && (!resize || k1 < nsmall / 2);
      int ki = ko;
      if (NO < NI) {          // restriction: drop the coarse Nyquist
        ok = ok && (k2 != -NO / 2);
        ki = k2 < 0 ? k2 + NI : k2;
      } else if (NO > NI) {   // prolongation: zero-pad, fine modes |k2| >= NI/2 vanish
        ok = ok && (k2 < NI / 2) && (k2 > -NI / 2);
        ki = k2 < 0 ? k2 + NI : k2;
      }
      float2 acc = make_float2(0.f, 0.f);
      if (ok) {
        for (int c = 0; c < a.nin; ++c) {
          const float2 sg = symbol(a, o, c, k1, k2);
          acc = cadd(acc, cmul(bin[c * P * NM + sw(l * NI + ki)], sg));
        }
        acc = cscale(acc, a.scale);
      }
      bout[sw(l * NO + ko)] = acc;
    }
    __syncthreads();
    fft_smem<LO, T, P, NT, true>(bout, a.tw_out);
    float2* dst = a.out + (long long)(g * a.nout + o) * a.out_fstride;
    for (int q = t; q < P * NO; q += NT) {
      const int l = q / NO, k2 = q % NO;
      const int k1 = line0 + l;
      if (k1 < a.nk1_out) dst[(long long)k1 * NO + k2] = bout[sw(q)];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side

// n = 2^L 3^T -> (L, T); L = -1 if n has another form
static void split_size(int n, int& L, int& T) {
  T = (n % 3 == 0) ? 1 : 0;
  int m = T ? n / 3 : n;
  L = 0;
  while ((1 << L) < m) ++L;
  if ((1 << L) != m) L = -1;
}

template <int L, int T>
static void launch_r2c(const float* in, long long fstride, float2* spec, long long sstride,
                       int n2, int F, const float2* tw, cudaStream_t st, const FieldMask& fm) {
  using C = RowCfg<L, T>;
  const size_t smem = (size_t)C::P * C::N * sizeof(float2);
  static_assert(C::P * C::N * sizeof(float2) <= 48 * 1024, "fits the default shared memory");
  dim3 grid(n2 / (2 * C::P), F);
  launch_k(k_rows_r2c<L, T>, dim3(grid), dim3(C::NT), smem, st, in, fstride, spec, sstride, n2, tw, fm);
}

template <int L, int T>
static void launch_c2r(const float2* spec, long long sstride, float* out, long long fstride,
                       const float* add, long long astride, int n2, int F, const float2* tw,
                       cudaStream_t st, const ChebEpilogue& cheb, const FieldMask& fm) {
  using C = RowCfg<L, T>;
  const size_t smem = (size_t)C::P * C::N * sizeof(float2);
  static_assert(C::P * C::N * sizeof(float2) <= 48 * 1024, "fits the default shared memory");
  dim3 grid(n2 / (2 * C::P), F);
  if (cheb.r)
    launch_k(k_rows_c2r<L, T, true>, dim3(grid), dim3(C::NT), smem, st, spec, sstride, out, fstride, add, astride, n2, tw, cheb, fm);
  else
    launch_k(k_rows_c2r<L, T, false>, dim3(grid), dim3(C::NT), smem, st, spec, sstride, out, fstride, add, astride, n2, tw, cheb, fm);
}

template <int LI, int LO, int T>
static void launch_cols(const ColArgs& a, int groups, cudaStream_t st) {
  using C = ColCfg<LI, LO, T>;
  const size_t smem = (size_t)(a.nin + 1) * C::P * C::NM * sizeof(float2);
  static_assert(3 * C::P * C::NM * sizeof(float2) <= 48 * 1024, "fits the default shared memory");
  static_assert((C::P * C::NM) % 128 == 0, "buffers start on multiples of 128 elements (sw)");
  dim3 grid((a.nk1_out + C::P - 1) / C::P, groups);
  launch_k(k_cols<LI, LO, T>, dim3(grid), dim3(C::NT), smem, st, a);
}

// supported line lengths: 2^L for L = 5..11, 3 * 2^L for L = 5..9 (96 .. 1536)
#define REGNK_SIZE_CASES(X) \
  X(5, 0) X(6, 0) X(7, 0) X(8, 0) X(9, 0) X(10, 0) X(11, 0) X(5, 1) X(6, 1) X(7, 1) X(8, 1) X(9, 1)
#define REGNK_RESTRICT_CASES(X) \
  X(6, 0) X(7, 0) X(8, 0) X(9, 0) X(10, 0) X(11, 0) X(6, 1) X(7, 1) X(8, 1) X(9, 1)
#define REGNK_PROLONG_CASES(X) \
  X(5, 0) X(6, 0) X(7, 0) X(8, 0) X(9, 0) X(10, 0) X(5, 1) X(6, 1) X(7, 1) X(8, 1)

bool fft_size_supported(int n) {
  int L, T;
  split_size(n, L, T);
  return L >= 5 && ((T == 0 && L <= 11) || (T == 1 && L <= 9));
}

void fft_rows_r2c(int n1, int n2, const float* in, long long fstride, float2* spec,
                  long long sstride, int F, const float2* tw, cudaStream_t st,
                  const FieldMask& fm) {
  int L, T;
  split_size(n1, L, T);
  switch (L * 2 + T) {
#define CASE(LL, TT) case LL * 2 + TT: launch_r2c<LL, TT>(in, fstride, spec, sstride, n2, F, tw, st, fm); break;
    REGNK_SIZE_CASES(CASE)
#undef CASE
    default: break;
  }
}

void fft_rows_c2r(int n1, int n2, const float2* spec, long long sstride, float* out,
                  long long fstride, const float* add, long long astride, int F,
                  const float2* tw, cudaStream_t st, const ChebEpilogue* cheb,
                  const FieldMask& fm) {
  int L, T;
  split_size(n1, L, T);
  const ChebEpilogue none;
  const ChebEpilogue& ce = cheb ? *cheb : none;
  switch (L * 2 + T) {
#define CASE(LL, TT) case LL * 2 + TT: launch_c2r<LL, TT>(spec, sstride, out, fstride, add, astride, n2, F, tw, st, ce, fm); break;
    REGNK_SIZE_CASES(CASE)
#undef CASE
    default: break;
  }
}

void fft_cols(const ColArgs& a, int groups, cudaStream_t st) {
  int li, ti, lo, to;
  split_size(a.n2_in, li, ti);
  split_size(a.n2_out, lo, to);
  if (ti != to) return;
  if (li == lo) {
    switch (li * 2 + ti) {
#define CASE(LL, TT) case LL * 2 + TT: launch_cols<LL, LL, TT>(a, groups, st); break;
      REGNK_SIZE_CASES(CASE)
#undef CASE
      default: break;
    }
  } else if (lo == li - 1) {
    switch (li * 2 + ti) {
#define CASE(LL, TT) case LL * 2 + TT: launch_cols<LL, LL - 1, TT>(a, groups, st); break;
      REGNK_RESTRICT_CASES(CASE)
#undef CASE
      default: break;
    }
  } else if (lo == li + 1) {
    switch (li * 2 + ti) {
#define CASE(LL, TT) case LL * 2 + TT: launch_cols<LL, LL + 1, TT>(a, groups, st); break;
      REGNK_PROLONG_CASES(CASE)
#undef CASE
      default: break;
    }
  }
}

// ---------------------------------------------------------------------------
// 3D grids: one pass of complex FFTs along one axis of F complex 3D arrays
// (x_1 fastest, `total` values each, `fstride` apart). The lines have length
// N and element stride `inner` (1 along x_1, n_1 along x_2, n_1 n_2 along
// x_3): element j of line (o, i) sits at (o N + j) inner + i. A block
// transforms P lines: consecutive o when inner = 1 (P N contiguous values),
// else consecutive i (P adjacent values per j, coalesced). Forward or
// inverse (unnormalised) Stockham passes as in the 2D kernels.
template <int L, int T, bool INV>
__global__ void __launch_bounds__(FftCfg<L, T>::NT)
k_axis(float2* __restrict__ z, long long fstride, long long inner, const float2* __restrict__ tw) {
  pdl_enter();
  constexpr int N = FftCfg<L, T>::N, P = FftCfg<L, T>::P, NT = FftCfg<L, T>::NT;
  extern __shared__ float2 sm[];
  float2* zf = z + (long long)blockIdx.y * fstride;
  const int t = threadIdx.x;
  long long o0 = 0, i0 = 0;
  if (inner == 1) {
    o0 = (long long)blockIdx.x * P;
  } else {
    const long long per = inner / P;
    o0 = blockIdx.x / per;
    i0 = (blockIdx.x % per) * P;
  }
  auto addr = [&](int l, int j) -> long long {
    return inner == 1 ? (o0 + l) * N + j : (o0 * N + j) * inner + i0 + l;
  };
  constexpr int LD = (P * N + NT - 1) / NT;
  float2 v[LD];
#pragma unroll
  for (int u = 0; u < LD; ++u) {
    const int q = t + u * NT;
    if ((P * N) % NT == 0 || q < P * N) {
      const int l = inner == 1 ? q / N : q % P, j = inner == 1 ? q % N : q / P;
      v[u] = zf[addr(l, j)];
    }
  }
#pragma unroll
  for (int u = 0; u < LD; ++u) {
    const int q = t + u * NT;
    if ((P * N) % NT == 0 || q < P * N) {
      const int l = inner == 1 ? q / N : q % P, j = inner == 1 ? q % N : q / P;
      sm[sw(l * N + j)] = v[u];
    }
  }
  __syncthreads();
  fft_smem<L, T, P, NT, INV>(sm, tw);
#pragma unroll
  for (int u = 0; u < LD; ++u) {
    const int q = t + u * NT;
    if ((P * N) % NT == 0 || q < P * N) {
      const int l = inner == 1 ? q / N : q % P, j = inner == 1 ? q % N : q / P;
      zf[addr(l, j)] = sm[sw(l * N + j)];
    }
  }
}

#define REGNK_AXIS_CASES(X) X(5, 0) X(6, 0) X(7, 0) X(8, 0) X(5, 1) X(6, 1)

bool fft_axis_supported(int n) {
  int L, T;
  split_size(n, L, T);
  return (T == 0 && L >= 5 && L <= 8) || (T == 1 && L >= 5 && L <= 6);
}

template <int L, int T>
static void launch_axis(float2* z, long long total, int F, long long inner, bool inverse,
                        const float2* tw, cudaStream_t st) {
  using C = FftCfg<L, T>;
  const size_t smem = (size_t)C::P * C::N * sizeof(float2);
  const long long lines = total / C::N;
  const dim3 grid((unsigned)(lines / C::P), F);
  if (inverse)
    launch_k(k_axis<L, T, true>, grid, dim3(C::NT), smem, st, z, total, inner, tw);
  else
    launch_k(k_axis<L, T, false>, grid, dim3(C::NT), smem, st, z, total, inner, tw);
}

void fft_axis(float2* z, long long total, int F, int n, long long inner, bool inverse,
              const float2* tw, cudaStream_t st) {
  int L, T;
  split_size(n, L, T);
  switch (L * 2 + T) {
#define CASE(LL, TT) case LL * 2 + TT: launch_axis<LL, TT>(z, total, F, inner, inverse, tw, st); break;
    REGNK_AXIS_CASES(CASE)
#undef CASE
    default: break;
  }
}

}  // namespace regnk
