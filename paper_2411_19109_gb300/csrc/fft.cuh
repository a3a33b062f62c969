// Shared-memory FFTs used by the demag convolution.
//
// fft_batch: `nseq` complex sequences of length L = 2^log2L, stored in
// shared memory at a fixed stride (L by default; a padded stride avoids bank
// conflicts on transposed loads), transformed by the whole thread block with a
// Stockham auto-sort schedule (radix-4 passes, one radix-2 pass when log2L
// is odd).  Each pass reads one buffer and writes the other, so no bit
// reversal is needed; the function returns the buffer holding the result.
// Twiddles come from a table of W_4096^k = exp(-2 pi i k/4096) computed in
// FP64 on the host (conjugated for the inverse transform).  The inverse is
// unnormalised; the 1/(Px Py) factor lives in the demag spectrum.
#pragma once

#include "common.cuh"

namespace llg {

// DIR = -1: forward (exp(-2 pi i jk/L)); DIR = +1: inverse, unnormalised.
template <typename C, int DIR>
__device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C a = cadd(x0, x2), b = csub(x0, x2);
  C c = cadd(x1, x3), d = csub(x1, x3);
  d = (DIR < 0) ? mul_mi(d) : mul_pi(d);
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}

template <typename C, int DIR>
__device__ __forceinline__ C twiddle(const C* __restrict__ tw, int m, int tstride) {
  C w = tw[m * tstride];
  if (DIR > 0) w.y = -w.y;
  return w;
}

template <typename C, int DIR>
__device__ C* fft_batch(C* a, C* b, int log2L, int nseq, const C* __restrict__ tw, int sstride = -1) {
  // sequence q starts at q * sstride (default: packed, sstride = L)
  const int L = 1 << log2L;
  if (sstride < 0) sstride = L;
  const int tstride = kTwiddleN >> log2L;
  const int tid = threadIdx.x, nt = blockDim.x;
  C* in = a;
  C* out = b;
  int rem = log2L, logNs = 0;
  while (rem >= 2) {
    const int Ns = 1 << logNs;
    const int quarter = L >> 2;
    const int lq = log2L - 2;
    const int tot = nseq << lq;
    const int tshift = log2L - logNs - 2;   // L/(4 Ns) = 2^tshift
    for (int t = tid; t < tot; t += nt) {
      const int q = t >> lq, j = t & (quarter - 1);
      const int base = q * sstride;
      const int k = j & (Ns - 1);
      C x0 = in[base + j], x1 = in[base + j + quarter];
      C x2 = in[base + j + 2 * quarter], x3 = in[base + j + 3 * quarter];
      if (logNs > 0) {
        const int m = k << tshift;
        x1 = cmul(x1, twiddle<C, DIR>(tw, m, tstride));
        x2 = cmul(x2, twiddle<C, DIR>(tw, 2 * m, tstride));
        x3 = cmul(x3, twiddle<C, DIR>(tw, 3 * m, tstride));
      }
      dft4<C, DIR>(x0, x1, x2, x3);
      const int d = base + ((j >> logNs) << (logNs + 2)) + k;
      out[d] = x0;
      out[d + Ns] = x1;
      out[d + 2 * Ns] = x2;
      out[d + 3 * Ns] = x3;
    }
    __syncthreads();
    C* s = in; in = out; out = s;
    rem -= 2;
    logNs += 2;
  }
  if (rem == 1) {
    const int Ns = 1 << logNs;
    const int half = L >> 1;
    const int lh = log2L - 1;
    const int tot = nseq << lh;
    const int tshift = log2L - logNs - 1;   // L/(2 Ns)
    for (int t = tid; t < tot; t += nt) {
      const int q = t >> lh, j = t & (half - 1);
      const int base = q * sstride;
      const int k = j & (Ns - 1);
      C x0 = in[base + j], x1 = in[base + j + half];
      if (logNs > 0) x1 = cmul(x1, twiddle<C, DIR>(tw, k << tshift, tstride));
      const int d = base + ((j >> logNs) << (logNs + 1)) + k;
      out[d] = cadd(x0, x1);
      out[d + Ns] = csub(x0, x1);
    }
    __syncthreads();
    C* s = in; in = out; out = s;
  }
  return in;
}

}  // namespace llg
