// Register-resident FFTs for the demag convolution.
//
// A length-L transform (L = 2^m, 8 <= L <= 2048) is computed by TT = L/8
// threads.  Thread t holds the eight elements x[t + TT*s], s = 0..7, on entry
// and X[t + TT*s] on exit (the same "stride-TT" layout, so global loads and
// stores of consecutive t are coalesced and no bit reversal is needed).
// The schedule is Stockham's auto-sort: one radix-2 or radix-4 pass first
// when m is not a multiple of 3, then radix-8 passes.  Between passes the
// data goes through shared memory, where index i lives at seq_pad(L, i) (pad
// slots spread the scattered writes over the banks); the last pass leaves
// its output in registers.
//
// Twiddles: W_L^m = tw[m * tws] for a table the caller provides (a copy of
// the FP64-computed W_4096^k table in shared memory, or the global table
// itself).  The double-float transforms instead read the per-pass table of
// fill_pass_twiddles (tws unused).  DIR = -1 is the forward transform, +1 the
// unnormalised inverse.
#pragma once

#include "common.cuh"

namespace llg {


template <typename C, int DIR>
__host__ __device__ __forceinline__ C rf_tw(const C* __restrict__ tw, int m, int stride) {
  C w = tw[m * stride];
  if (DIR > 0) w.y = -w.y;
  return w;
}

template <typename C, int DIR>
__host__ __device__ __forceinline__ void rf_dft2(C& a, C& b) {
  const C s = cadd(a, b), d = csub(a, b);
  a = s;
  b = d;
}

template <typename C, int DIR>
__host__ __device__ __forceinline__ void rf_dft4(C& x0, C& x1, C& x2, C& x3) {
  C a = cadd(x0, x2), b = csub(x0, x2);
  C c = cadd(x1, x3), d = csub(x1, x3);
  d = (DIR < 0) ? mul_mi(d) : mul_pi(d);
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}

// 8-point DFT in place: x[k] <- sum_j x[j] W_8^{jk} (the four sums, then
// the four differences: in the double-float passes this order spilled less)
template <typename C, int DIR>
__host__ __device__ __forceinline__ void rf_dft8(C x[8]) {
  using R = decltype(C::x);
  const R h = (R)0.70710678118654752440;
  C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  rf_dft4<C, DIR>(e0, e1, e2, e3);
  rf_dft4<C, DIR>(o0, o1, o2, o3);
  // o_k *= W_8^k
  if (DIR < 0) {
    o1 = mk<C>(h * (o1.x + o1.y), h * (o1.y - o1.x));      // (1 - i)/sqrt2
    o2 = mul_mi(o2);
    o3 = mk<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y));     // (-1 - i)/sqrt2
  } else {
    o1 = mk<C>(h * (o1.x - o1.y), h * (o1.x + o1.y));      // (1 + i)/sqrt2
    o2 = mul_pi(o2);
    o3 = mk<C>(-h * (o3.x + o3.y), h * (o3.x - o3.y));     // (-1 + i)/sqrt2
  }
  x[0] = cadd(e0, o0);
  x[1] = cadd(e1, o1);
  x[2] = cadd(e2, o2);
  x[3] = cadd(e3, o3);
  x[4] = csub(e0, o0);
  x[5] = csub(e1, o1);
  x[6] = csub(e2, o2);
  x[7] = csub(e3, o3);
}

// DFTs of 4 and 8 points whose upper half of inputs is zero (x2 = x3 = 0,
// x4..x7 = 0): the first pass of a forward transform of zero-padded data.
// Same values as rf_dft4 / rf_dft8 on those inputs, up to the sign of zero
// results; the additions of the zeros are left out.  The double-float passes
// need this spelled out: a compensated sum with a zero operand is not
// something the compiler may fold (it could change the sign of a zero).
template <typename C, int DIR>
__host__ __device__ __forceinline__ void rf_dft4_half(C& x0, C& x1, C& x2, C& x3) {
  const C a = x0, c = x1;
  const C d = (DIR < 0) ? mul_mi(c) : mul_pi(c);
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(a, d);
  x3 = csub(a, d);
}
template <typename C, int DIR>
__host__ __device__ __forceinline__ void rf_dft8_half(C x[8]) {
  using R = decltype(C::x);
  const R h = (R)0.70710678118654752440;
  C e0 = x[0], e1 = x[2], e2, e3;
  C o0 = x[1], o1 = x[3], o2, o3;
  rf_dft4_half<C, DIR>(e0, e1, e2, e3);
  rf_dft4_half<C, DIR>(o0, o1, o2, o3);
  if (DIR < 0) {
    o1 = mk<C>(h * (o1.x + o1.y), h * (o1.y - o1.x));
    o2 = mul_mi(o2);
    o3 = mk<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  } else {
    o1 = mk<C>(h * (o1.x - o1.y), h * (o1.x + o1.y));
    o2 = mul_pi(o2);
    o3 = mk<C>(-h * (o3.x + o3.y), h * (o3.x - o3.y));
  }
  x[0] = cadd(e0, o0);
  x[4] = csub(e0, o0);
  x[1] = cadd(e1, o1);
  x[5] = csub(e1, o1);
  x[2] = cadd(e2, o2);
  x[6] = csub(e2, o2);
  x[3] = cadd(e3, o3);
  x[7] = csub(e3, o3);
}

// First pass (stage size 1, no twiddles) of radix RP when the inputs of
// slots s >= 4 are zero: butterfly b takes v[b + r*(8/RP)], which is zero
// exactly for r >= RP/2.  Same outputs and destinations as
// rf_pass<C, L, RP, DIR>(v, t, 1, ...) on such inputs.
template <typename C, int L, int RP, int DIR>
__host__ __device__ __forceinline__ void rf_pass_half(C v[8], int t, int dst[8]) {
  constexpr int TT = L / 8;
  constexpr int NB = 8 / RP;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = t + TT * b;
    C x[RP];
#pragma unroll
    for (int r = 0; r < RP / 2; ++r) x[r] = v[b + r * NB];
    if constexpr (RP == 2) {
      x[1] = x[0];
    } else if constexpr (RP == 4) {
      rf_dft4_half<C, DIR>(x[0], x[1], x[2], x[3]);
    } else {
      rf_dft8_half<C, DIR>(x);
    }
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      v[b + r * NB] = x[r];
      dst[b + r * NB] = j * RP + r;
    }
  }
}

// One Stockham pass of radix RP on the eight registers of thread t.
// Butterfly b of the thread is j = t + TT*b (b < 8/RP); its inputs are
// v[b + r*(8/RP)], r < RP.  Returns the outputs in the same slots; `dst`
// receives the shared-memory index of each slot's output.
template <typename C, int L, int RP, int DIR>
__host__ __device__ __forceinline__ void rf_pass(C v[8], int t, int Ns, const C* __restrict__ tw, int tws, int dst[8]) {
  constexpr int TT = L / 8;
  constexpr int NB = 8 / RP;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = t + TT * b;
    const int k = j & (Ns - 1);
    const int step = (L / (Ns * RP)) * k;         // twiddle W_L^{r*step}
    C x[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) x[r] = v[b + r * NB];
    if (Ns > 1) {
      using R = decltype(C::x);
      if constexpr (sizeof(R) == 4 && RP >= 4) {
        // FP32: load W^step only and form its powers by products (at most
        // three roundings deep, ~3 ulp), trading shared-memory loads, the
        // limiting resource of these kernels, for FMAs
        C w[RP];
        w[1] = rf_tw<C, DIR>(tw, step, tws);
        w[2] = cmul(w[1], w[1]);
        w[3] = cmul(w[2], w[1]);
        if constexpr (RP == 8) {
          w[4] = cmul(w[2], w[2]);
          w[5] = cmul(w[4], w[1]);
          w[6] = cmul(w[3], w[3]);
          w[7] = cmul(w[4], w[3]);
        }
#pragma unroll
        for (int r = 1; r < RP; ++r) x[r] = cmul(x[r], w[r]);
      } else {
#pragma unroll
        for (int r = 1; r < RP; ++r) x[r] = cmul(x[r], rf_tw<C, DIR>(tw, r * step, tws));
      }
    }
    if (RP == 2) {
      rf_dft2<C, DIR>(x[0], x[1]);
    } else if (RP == 4) {
      rf_dft4<C, DIR>(x[0], x[1], x[2], x[3]);
    } else {
      rf_dft8<C, DIR>(x);
    }
    const int base = (j / Ns) * Ns * RP + k;
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      v[b + r * NB] = x[r];
      dst[b + r * NB] = base + r * Ns;
    }
  }
}

__host__ __device__ constexpr int log2_len(int L) {
  return (L == 8) ? 3 : (L == 16) ? 4 : (L == 32) ? 5 : (L == 64) ? 6 : (L == 128) ? 7 : (L == 256) ? 8
       : (L == 512) ? 9 : (L == 1024) ? 10 : 11;
}
// log2 of the stage size after the first pass of a length-L transform.
__host__ __device__ constexpr int first_pass_lns(int L) { return log2_len(L) % 3 == 1 ? 1 : (log2_len(L) % 3 == 2 ? 2 : 3); }

// Per-pass twiddles of the rolled radix-8 passes.  The pass of stage size
// Ns = 2^lns multiplies input r of butterfly k = t mod Ns by W_L^{r k L/(8 Ns)},
// r = 1..7; its table holds these at [7 k + r - 1].  Lanes with distinct k
// then read 16-byte entries 7 apart (distinct bank groups), lanes with equal
// k one address.  The tables of the passes follow each other, first pass
// excluded (no twiddles at Ns = 1): 7 (Ns_1 + Ns_2 + ...) < L entries.
// Entries i0, i0 + di, ... are filled (one call per thread of a block, or a
// single host call with i0 = 0, di = 1).
template <typename C, int L>
__host__ __device__ __forceinline__ void fill_pass_twiddles(C* dst, const C* __restrict__ tw4096, int i0, int di) {
  constexpr int M = log2_len(L);
  int off = 0;
  for (int lns = first_pass_lns(L); lns < M; lns += 3) {
    const int n = 7 << lns;
    for (int i = i0; i < n; i += di) {
      const int k = i / 7, r = i - 7 * k + 1;
      dst[off + i] = tw4096[(r * (k << (M - lns - 3))) * (kTwiddleN / L)];
    }
    off += n;
  }
}

// A radix-8 Stockham pass with the stage size Ns = 2^lns a run-time value
// (shifts in place of the divisions by Ns), for the rolled pass loop of the
// double-float transforms; same data movement as rf_pass<C, L, 8, DIR> at
// Ns > 1, twiddles from this pass's table twp of fill_pass_twiddles.
template <typename C, int L, int DIR>
__host__ __device__ __forceinline__ void rf_pass8_rt(C v[8], int t, int lns, const C* __restrict__ twp, int dst[8]) {
  const int k = t & ((1 << lns) - 1);
  C x[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) x[r] = v[r];
#pragma unroll
  for (int r = 1; r < 8; ++r) x[r] = cmul(x[r], rf_tw<C, DIR>(twp, 7 * k + r - 1, 1));
  rf_dft8<C, DIR>(x);
  const int base = ((t >> lns) << (lns + 3)) + k;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    v[r] = x[r];
    dst[r] = base + (r << lns);
  }
}

// Where slot s of thread t goes after pass p - 1 of a rolled transform: after
// the first pass (radix R0 = 8 / NB, stage size 1) butterfly t + TT (s mod NB)
// writes its output s / NB to (t + TT (s mod NB)) R0 + s / NB; after a rolled
// radix-8 pass of stage size 2^pl butterfly t writes output s to
// rf_pass8_rt's destination.  pl is the stage size's log2 of pass p - 1 for
// p >= 2 (unused for p == 1).
template <int L>
__host__ __device__ __forceinline__ int rolled_exchange_dst(int p, int pl, int t, int s) {
  constexpr int TT = L / 8;
  constexpr int R0 = 1 << first_pass_lns(L);
  constexpr int NB0 = 8 / R0;
  if (p == 1) return (t + TT * (s % NB0)) * R0 + s / NB0;
  return (((t >> pl) << (pl + 3)) | (t & ((1 << pl) - 1))) + (s << pl);
}

template <typename C> struct RolledPasses { static constexpr bool value = false; };
template <> struct RolledPasses<dcplx> { static constexpr bool value = true; };

// Synchronisation of the threads that exchange one sequence: the whole block,
// one warp (the group lies inside it), or a named barrier over `n` threads.
struct GroupSync {
  int id;            // 0: whole block; < 0: the group's lanes of one warp; > 0: named barrier id
  int n;             // threads in the named barrier
  unsigned mask;     // id < 0: the lanes of the group
  __device__ __forceinline__ void operator()() const {
    if (id == 0) {
      __syncthreads();
    } else if (id < 0) {
      __syncwarp(mask);
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
  }
};

// Group sync for groups of TT consecutive threads (group index tid / TT):
// the group's own lanes of its warp when a group fits in a warp, a named
// barrier otherwise.  Either way only the group's threads take part, so a
// group may skip a transform while other groups of its warp or block run one.
__device__ __forceinline__ GroupSync group_sync(int TT) {
  GroupSync g;
  g.mask = 0xffffffffu;
  if (TT <= 32) {
    g.id = -1;
    g.n = 32;
    if (TT < 32) g.mask = ((1u << TT) - 1u) << ((threadIdx.x & 31) / TT * TT);
  } else {
    g.id = 1 + (int)(threadIdx.x / TT);
    g.n = TT;
  }
  return g;
}

// Full transform of NCOMP sequences held by the same threads (v[c][8] for
// c < NCOMP).  Element i of sequence c is exchanged through
// sm[(c*sstride + pad(i)) * estride]: estride = 1 keeps each sequence
// contiguous, estride = G interleaves G groups element by element (lanes of
// consecutive groups then touch consecutive banks).  Every thread of the
// block must call it (it synchronises the block between passes).
// HALF_IN: the caller guarantees v[c][s] == 0 for s >= 4 (the upper half of a
// zero-padded sequence); the double-float first pass then skips the zeros.
template <typename C, int L, int DIR, int NCOMP, bool HALF_IN = false>
__device__ __forceinline__ void regfft(C (&v)[NCOMP][8], C* sm, int sstride, int estride, int t,
                                       const C* __restrict__ tw, int tws, GroupSync sync = GroupSync{0, 0}) {
  constexpr int M = (L == 8) ? 3 : (L == 16) ? 4 : (L == 32) ? 5 : (L == 64) ? 6 : (L == 128) ? 7
                  : (L == 256) ? 8 : (L == 512) ? 9 : (L == 1024) ? 10 : 11;
  static_assert((1 << M) == L, "L must be a power of two in [8, 2048]");
  constexpr int TT = L / 8;
  constexpr int R0 = (M % 3 == 1) ? 2 : (M % 3 == 2) ? 4 : 8;
  constexpr int NPASS = (M % 3 == 0) ? M / 3 : M / 3 + 1;
  int dst[8];
  if constexpr (RolledPasses<C>::value) {
    // double-float: the first pass, then one copy of the radix-8 pass code
    // in a rolled loop (a double-float butterfly is ~10x the code of an FP32
    // one, and the unrolled passes overflowed the instruction cache)
#pragma unroll
    for (int c = 0; c < NCOMP; ++c) {   // Ns = 1: no twiddles
      if constexpr (HALF_IN) rf_pass_half<C, L, R0, DIR>(v[c], t, dst);
      else rf_pass<C, L, R0, DIR>(v[c], t, 1, tw, tws, dst);
    }
    // The exchange recomputes each slot's write index from t
    // (rolled_exchange_dst) rather than carrying the eight indices across the
    // pass in registers.
    int lns = first_pass_lns(L);
    const C* twp = tw;
#pragma unroll 1
    for (int p = 1; p < NPASS; ++p) {
#pragma unroll
      for (int c = 0; c < NCOMP; ++c)
#pragma unroll
        for (int s = 0; s < 8; ++s)
          sm[(c * sstride + seq_pad<C>(L, rolled_exchange_dst<L>(p, lns - 3, t, s))) * estride] = v[c][s];
      sync();
#pragma unroll
      for (int c = 0; c < NCOMP; ++c)
#pragma unroll
        for (int s = 0; s < 8; ++s) v[c][s] = sm[(c * sstride + seq_pad<C>(L, t + TT * s)) * estride];
      sync();
#pragma unroll
      for (int c = 0; c < NCOMP; ++c) rf_pass8_rt<C, L, DIR>(v[c], t, lns, twp, dst);
      twp += 7 << lns;
      lns += 3;
    }
    return;
  }
  int Ns = 1;
#pragma unroll
  for (int p = 0; p < NPASS; ++p) {
    if (p > 0) {
      // exchange: scattered write of the previous pass, then the strided read
#pragma unroll
      for (int c = 0; c < NCOMP; ++c)
#pragma unroll
        for (int s = 0; s < 8; ++s) sm[(c * sstride + seq_pad<C>(L, dst[s])) * estride] = v[c][s];
      sync();
#pragma unroll
      for (int c = 0; c < NCOMP; ++c)
#pragma unroll
        for (int s = 0; s < 8; ++s) v[c][s] = sm[(c * sstride + seq_pad<C>(L, t + TT * s)) * estride];
      sync();
    }
    if (p == 0 && R0 == 2) {
#pragma unroll
      for (int c = 0; c < NCOMP; ++c) rf_pass<C, L, 2, DIR>(v[c], t, Ns, tw, tws, dst);
      Ns *= 2;
    } else if (p == 0 && R0 == 4) {
#pragma unroll
      for (int c = 0; c < NCOMP; ++c) rf_pass<C, L, 4, DIR>(v[c], t, Ns, tw, tws, dst);
      Ns *= 4;
    } else {
#pragma unroll
      for (int c = 0; c < NCOMP; ++c) rf_pass<C, L, 8, DIR>(v[c], t, Ns, tw, tws, dst);
      Ns *= 8;
    }
  }
}

// ---------------------------------------------------------------------------
// 16 elements per thread (TT = L/16 threads per sequence): radix-16 passes,
// so L = 128, 256 take one shared-memory exchange instead of two and
// L = 1024 two instead of three.  Same stride layout: thread t holds element
// t + TT*s in v[s] on entry and on exit.
// ---------------------------------------------------------------------------

// a * W_16^M with W_16 = exp(DIR * 2 pi i / 16) (DIR = -1 forward), M fixed.
template <typename C, int DIR, int M>
__host__ __device__ __forceinline__ C rf_w16(C a) {
  using R = decltype(C::x);
  constexpr int m = M & 15;
  const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173, h = (R)0.70710678118654752440;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (m == 4) {
    return DIR < 0 ? mul_mi(a) : mul_pi(a);
  } else if constexpr (m == 8) {
    return mk<C>(-a.x, -a.y);
  } else if constexpr (m == 12) {
    return DIR < 0 ? mul_pi(a) : mul_mi(a);
  } else {
    // cos and sin of 2 pi m / 16
    const R cs = (m == 1 || m == 15) ? c1 : (m == 2 || m == 14) ? h : (m == 3 || m == 13) ? s1
               : (m == 5 || m == 11) ? -s1 : (m == 6 || m == 10) ? -h : -c1;
    const R sn = (m == 1 || m == 7) ? s1 : (m == 2 || m == 6) ? h : (m == 3 || m == 5) ? c1
               : (m == 9 || m == 15) ? -s1 : (m == 10 || m == 14) ? -h : -c1;
    const R wy = DIR < 0 ? -sn : sn;
    return mk<C>(a.x * cs - a.y * wy, a.x * wy + a.y * cs);
  }
}

// 16-point DFT in place as 4 x 4: x[k1 + 4 k2] = sum_n2 W16^{n2 k1} W4^{n2 k2}
// sum_n1 W4^{n1 k1} x[4 n1 + n2].
template <typename C, int DIR>
__host__ __device__ __forceinline__ void rf_dft16(C x[16]) {
  C a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C y0 = x[n2], y1 = x[4 + n2], y2 = x[8 + n2], y3 = x[12 + n2];
    rf_dft4<C, DIR>(y0, y1, y2, y3);
    a[n2][0] = y0; a[n2][1] = y1; a[n2][2] = y2; a[n2][3] = y3;
  }
  a[1][1] = rf_w16<C, DIR, 1>(a[1][1]);
  a[1][2] = rf_w16<C, DIR, 2>(a[1][2]);
  a[1][3] = rf_w16<C, DIR, 3>(a[1][3]);
  a[2][1] = rf_w16<C, DIR, 2>(a[2][1]);
  a[2][2] = rf_w16<C, DIR, 4>(a[2][2]);
  a[2][3] = rf_w16<C, DIR, 6>(a[2][3]);
  a[3][1] = rf_w16<C, DIR, 3>(a[3][1]);
  a[3][2] = rf_w16<C, DIR, 6>(a[3][2]);
  a[3][3] = rf_w16<C, DIR, 9>(a[3][3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C z0 = a[0][k1], z1 = a[1][k1], z2 = a[2][k1], z3 = a[3][k1];
    rf_dft4<C, DIR>(z0, z1, z2, z3);
    x[k1] = z0; x[k1 + 4] = z1; x[k1 + 8] = z2; x[k1 + 12] = z3;
  }
}

// One Stockham pass of radix RP on the sixteen registers of thread t
// (butterfly b: j = t + TT*b, inputs v[b + r*(16/RP)]).
template <typename C, int L, int RP, int DIR>
__host__ __device__ __forceinline__ void rf_pass16(C v[16], int t, int Ns, const C* __restrict__ tw, int tws,
                                          const C* __restrict__ tw4, int dst[16]) {
  constexpr int TT = L / 16;
  constexpr int NB = 16 / RP;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = t + TT * b;
    const int k = j & (Ns - 1);
    const int step = (L / (Ns * RP)) * k;         // twiddle W_L^{r*step}
    C x[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) x[r] = v[b + r * NB];
    if (Ns > 1) {
      using R = decltype(C::x);
      if constexpr (sizeof(R) == 4 && RP == 16) {
        // FP32: W^step and W^{4 step} loaded (the latter from its own
        // contiguous table when given: tw4[k] = W^{4k}, k < L/16), the other
        // powers by products at most three roundings deep
        C w[16];
        w[1] = rf_tw<C, DIR>(tw, step, tws);
        w[4] = tw4 ? rf_tw<C, DIR>(tw4, step, 1) : rf_tw<C, DIR>(tw, 4 * step, tws);
        w[2] = cmul(w[1], w[1]);
        w[3] = cmul(w[2], w[1]);
        w[5] = cmul(w[4], w[1]);
        w[6] = cmul(w[4], w[2]);
        w[7] = cmul(w[4], w[3]);
        w[8] = cmul(w[4], w[4]);
        w[9] = cmul(w[8], w[1]);
        w[10] = cmul(w[8], w[2]);
        w[11] = cmul(w[8], w[3]);
        w[12] = cmul(w[8], w[4]);
        w[13] = cmul(w[12], w[1]);
        w[14] = cmul(w[12], w[2]);
        w[15] = cmul(w[12], w[3]);
#pragma unroll
        for (int r = 1; r < RP; ++r) x[r] = cmul(x[r], w[r]);
      } else {
#pragma unroll
        for (int r = 1; r < RP; ++r) x[r] = cmul(x[r], rf_tw<C, DIR>(tw, r * step, tws));
      }
    }
    if constexpr (RP == 2) {
      rf_dft2<C, DIR>(x[0], x[1]);
    } else if constexpr (RP == 4) {
      rf_dft4<C, DIR>(x[0], x[1], x[2], x[3]);
    } else if constexpr (RP == 8) {
      rf_dft8<C, DIR>(x);
    } else {
      rf_dft16<C, DIR>(x);
    }
    const int base = (j / Ns) * Ns * RP + k;
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      v[b + r * NB] = x[r];
      dst[b + r * NB] = base + r * Ns;
    }
  }
}

// Full transform of one sequence held 16 elements per thread; element i is
// exchanged through sm[map(i)] (map: a permutation of [0, L) into the
// group's shared-memory slots).  First pass radix 2^(log2 L mod 4) (16 when
// that is 0), then radix-16 passes.  tw4: optional table of W_L^{4k}.
template <typename C, int L, int DIR, typename Map>
__device__ __forceinline__ void regfft16(C (&v)[16], C* sm, int t, const C* __restrict__ tw, int tws,
                                         const C* __restrict__ tw4, const Map& map, GroupSync sync) {
  constexpr int M = (L == 16) ? 4 : (L == 32) ? 5 : (L == 64) ? 6 : (L == 128) ? 7 : (L == 256) ? 8
                  : (L == 512) ? 9 : (L == 1024) ? 10 : 11;
  static_assert((1 << M) == L, "L must be a power of two in [16, 2048]");
  constexpr int TT = L / 16;
  constexpr int R0 = (M % 4 == 0) ? 16 : (1 << (M % 4));
  constexpr int NPASS = (M % 4 == 0) ? M / 4 : M / 4 + 1;
  int dst[16];
  int Ns = 1;
#pragma unroll
  for (int p = 0; p < NPASS; ++p) {
    if (p > 0) {
#pragma unroll
      for (int s = 0; s < 16; ++s) sm[map(dst[s])] = v[s];
      sync();
#pragma unroll
      for (int s = 0; s < 16; ++s) v[s] = sm[map(t + TT * s)];
      sync();
    }
    if (p == 0) {
      rf_pass16<C, L, R0, DIR>(v, t, Ns, tw, tws, tw4, dst);
      Ns *= R0;
    } else {
      rf_pass16<C, L, 16, DIR>(v, t, Ns, tw, tws, tw4, dst);
      Ns *= 16;
    }
  }
}

// Copy W_P^k, k < P, from the global W_4096 table into shared memory
// (all threads; the caller synchronises before use).
template <typename C>
__device__ __forceinline__ void load_twiddles(C* dst, const C* __restrict__ tw4096, int P) {
  const int stride = kTwiddleN / P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) dst[i] = tw4096[i * stride];
}

}  // namespace llg
