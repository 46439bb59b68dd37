// Shared definitions of the sm_103a kernels and the host runtime.
//
// Field layout: a scalar field on an n1 x n2 periodic grid is n1*n2 float32,
// row-major with x_1 fastest (u[j*n1 + i]); a vector field is its two
// components back to back. Spectra are stored "column major": the half
// spectrum of a real field has (n1/2 + 1) lines, one per k1 >= 0, each line
// holding the n2 complex coefficients over k2 contiguously. This makes both
// FFT passes read and write whole contiguous lines.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

#define REG_HD __host__ __device__ __forceinline__

namespace regnk {

struct GridDims {
  int n1, n2;        // nodes per axis (2^k or 3 * 2^k, multiples of 32)
  int log1, log2;    // log2 of n1, n2 if powers of two, else -1
  long long N;       // n1 * n2
  int nk1;           // n1 / 2 + 1 spectral lines
  long long spec;    // nk1 * n2 complex values per spectrum
};

inline GridDims make_grid(int n1, int n2) {
  GridDims g;
  g.n1 = n1;
  g.n2 = n2;
  g.log1 = 0;
  while ((1 << g.log1) < n1) ++g.log1;
  if ((1 << g.log1) != n1) g.log1 = -1;
  g.log2 = 0;
  while ((1 << g.log2) < n2) ++g.log2;
  if ((1 << g.log2) != n2) g.log2 = -1;
  g.N = (long long)n1 * n2;
  g.nk1 = n1 / 2 + 1;
  g.spec = (long long)g.nk1 * n2;
  return g;
}

// Signed wavenumber of FFT index k on an n-point grid.
REG_HD int signed_k(int k, int n) { return k < n / 2 ? k : k - n; }

// Periodic wrap of an index known to lie in [-n, 2n).
REG_HD int wrap_once(int i, int n) {
  i = i < 0 ? i + n : i;
  return i >= n ? i - n : i;
}

}  // namespace regnk
