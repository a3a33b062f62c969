// Host driver for the register FFT passes of csrc/regfft.cuh (compiled for
// the host by tests/test_fft_host.py; no GPU).  For each length L, lane width
// (8 or 16 elements per thread), precision and direction it runs the passes
// in the schedule regfft / regfft16 use: thread t holds x[t + TT s], each pass
// leaves its outputs with their destination indices, and the exchange writes
// them to those slots and reads back x[t + TT s].  It prints, per case, the
// relative L2 error against a direct DFT in long double and whether every
// pass scattered to a permutation of [0, L) (so no two lanes write one slot).
// Precisions: FP32, FP64 and double-float (dcplx, the adjoint's frequency
// domain option).
#include <cmath>
#include <cstdio>
#include <vector>

#include "regfft.cuh"

using namespace llg;

// FP32 operations of the double-float arithmetic (dfloat.cuh counts them in
// this host build, compiled with LLG_HOST_COUNT_OPS)
unsigned long long llg_host_fp32_ops = 0;

// value of a real part as long double, for the comparison
static long double to_ld(float v) { return v; }
static long double to_ld(double v) { return v; }
static long double to_ld(dfloat v) { return (long double)v.hi + (long double)v.lo; }

static double lcg_unit(unsigned long long& s) {
  s = s * 6364136223846793005ULL + 1442695040888963407ULL;
  return (double)(s >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

template <typename C>
static std::vector<C> twiddles() {
  std::vector<C> tw(kTwiddleN);
  for (int k = 0; k < kTwiddleN; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)kTwiddleN;
    tw[k].x = (decltype(C::x))std::cos(ang);
    tw[k].y = (decltype(C::x))std::sin(ang);
  }
  return tw;
}

constexpr int log2i(int L) { return L <= 1 ? 0 : 1 + log2i(L / 2); }

// Runs one pass of radix RP over all threads; returns false if the
// destinations are not a permutation of [0, L).
// (the double-float transforms run their radix-8 passes after the first
// through rf_pass8_rt, with the stage size as a run-time shift and the
// twiddles from the per-pass table of fill_pass_twiddles)
template <typename C, int L, int W, int RP, int DIR>
static bool pass(std::vector<C>& v, std::vector<int>& dst, int Ns, const C* tw, const C* tw4) {
  constexpr int TT = L / W;
  int lns = 0;
  while ((1 << lns) < Ns) ++lns;
  std::vector<C> ptab;
  int poff = 0;
  if constexpr (W == 8 && RP == 8 && RolledPasses<C>::value) {
    ptab.resize(L);
    fill_pass_twiddles<C, L>(ptab.data(), tw, 0, 1);
    for (int l = first_pass_lns(L); l < lns; l += 3) poff += 7 << l;
  }
  for (int t = 0; t < TT; ++t) {
    if constexpr (W == 8 && RP == 8 && RolledPasses<C>::value) {
      if (Ns > 1) {
        rf_pass8_rt<C, L, DIR>(&v[t * W], t, lns, ptab.data() + poff, &dst[t * W]);
        continue;
      }
    }
    if constexpr (W == 8)
      rf_pass<C, L, RP, DIR>(&v[t * W], t, Ns, tw, kTwiddleN / L, &dst[t * W]);
    else
      rf_pass16<C, L, RP, DIR>(&v[t * W], t, Ns, tw, kTwiddleN / L, tw4, &dst[t * W]);
  }
  std::vector<int> seen(L, 0);
  for (int i = 0; i < L; ++i) {
    if (dst[i] < 0 || dst[i] >= L || seen[dst[i]]++) return false;
  }
  // the double-float transforms recompute these destinations at the next
  // exchange (rolled_exchange_dst) instead of keeping them
  if constexpr (W == 8) {
    const int p = Ns == 1 ? 1 : 2;
    for (int t = 0; t < TT; ++t)
      for (int s = 0; s < W; ++s)
        if (rolled_exchange_dst<L>(p, lns, t, s) != dst[t * W + s]) return false;
  }
  return true;
}

template <typename C, int L, int W, int DIR>
static void run(const char* name, bool with_tw4) {
  constexpr int TT = L / W;
  constexpr int M = log2i(L);
  constexpr int LB = W == 8 ? 3 : 4;                       // log2 of the full radix
  constexpr int R0 = (M % LB == 0) ? W : (1 << (M % LB));
  constexpr int NPASS = (M % LB == 0) ? M / LB : M / LB + 1;
  const std::vector<C> tw = twiddles<C>();
  std::vector<C> tw4(L / 16 > 0 ? L / 16 : 1);
  for (int k = 0; k < L / 16; ++k) tw4[k] = tw[(4 * k * (kTwiddleN / L)) % kTwiddleN];
  unsigned long long seed = 0x9E3779B97F4A7C15ULL ^ (unsigned long long)(L * 131 + W * 7 + (DIR > 0));
  std::vector<long double> xr(L), xi(L);
  std::vector<C> v(L);
  for (int i = 0; i < L; ++i) {
    const double a = lcg_unit(seed), b = lcg_unit(seed);
    v[(i % TT) * W + i / TT].x = (decltype(C::x))a;      // x[t + TT s] -> thread t, slot s
    v[(i % TT) * W + i / TT].y = (decltype(C::x))b;
    xr[i] = to_ld(v[(i % TT) * W + i / TT].x);
    xi[i] = to_ld(v[(i % TT) * W + i / TT].y);
  }
  std::vector<int> dst(L);
  bool perm = true;
  int Ns = 1;
  for (int p = 0; p < NPASS; ++p) {
    if (p > 0) {                                           // the shared-memory exchange
      std::vector<C> sm(L);
      for (int i = 0; i < L; ++i) sm[dst[i]] = v[i];
      for (int t = 0; t < TT; ++t)
        for (int s = 0; s < W; ++s) v[t * W + s] = sm[t + TT * s];
    }
    const C* t4 = with_tw4 ? tw4.data() : nullptr;
    if (p == 0 && R0 == 2) {
      perm &= pass<C, L, W, 2, DIR>(v, dst, Ns, tw.data(), t4);
      Ns *= 2;
    } else if (p == 0 && R0 == 4) {
      perm &= pass<C, L, W, 4, DIR>(v, dst, Ns, tw.data(), t4);
      Ns *= 4;
    } else if (p == 0 && R0 == 8 && W == 16) {
      perm &= pass<C, L, W, 8, DIR>(v, dst, Ns, tw.data(), t4);
      Ns *= 8;
    } else {
      perm &= pass<C, L, W, W, DIR>(v, dst, Ns, tw.data(), t4);
      Ns *= W;
    }
  }
  // outputs: X[t + TT s] in thread t, slot s (the last pass leaves them in registers)
  std::vector<long double> cr(L), ci(L);
  for (int m = 0; m < L; ++m) {
    const long double ang = (long double)DIR * 2.0L * 3.14159265358979323846264338327950288L * (long double)m /
                            (long double)L;
    cr[m] = cosl(ang);
    ci[m] = sinl(ang);
  }
  long double num = 0, den = 0;
  for (int k = 0; k < L; ++k) {
    long double sr = 0, si = 0;
    for (int j = 0; j < L; ++j) {
      const int m = (int)((long long)j * k % L);
      const long double c = cr[m], s = ci[m];
      sr += xr[j] * c - xi[j] * s;
      si += xr[j] * s + xi[j] * c;
    }
    int idx = -1;
    for (int i = 0; i < L; ++i)
      if (dst[i] == k) idx = i;                            // slot holding X[k]
    const long double er = to_ld(v[idx].x) - sr, ei = to_ld(v[idx].y) - si;
    num += er * er + ei * ei;
    den += sr * sr + si * si;
  }
  std::printf("%s %d %d %d %d %.3e %d\n", name, W, L, DIR, with_tw4 ? 1 : 0, (double)sqrtl(num / den),
              perm ? 1 : 0);
}

template <typename C, int W>
static void all_lengths(const char* name) {
  if constexpr (W == 8) {
    run<C, 8, W, -1>(name, false);
    run<C, 8, W, +1>(name, false);
  }
  run<C, 16, W, -1>(name, false);
  run<C, 16, W, +1>(name, false);
  run<C, 32, W, -1>(name, false);
  run<C, 32, W, +1>(name, false);
  run<C, 64, W, -1>(name, false);
  run<C, 64, W, +1>(name, false);
  run<C, 128, W, -1>(name, false);
  run<C, 128, W, +1>(name, false);
  run<C, 256, W, -1>(name, false);
  run<C, 256, W, +1>(name, false);
  run<C, 512, W, -1>(name, false);
  run<C, 512, W, +1>(name, false);
  run<C, 1024, W, -1>(name, false);
  run<C, 1024, W, +1>(name, false);
  run<C, 2048, W, -1>(name, false);
  run<C, 2048, W, +1>(name, false);
  if constexpr (W == 16) {
    run<C, 128, W, -1>(name, true);
    run<C, 256, W, +1>(name, true);
    run<C, 1024, W, -1>(name, true);
    run<C, 1024, W, +1>(name, true);
  }
}

// The first pass of a zero-padded forward transform in its half-input form
// (rf_pass_half: inputs of slots s >= 4 known to be zero) must give the
// values and destinations of the full first pass on such inputs (a zero
// result may differ in sign only, which == ignores).  Prints
// "half <prec> <L> <DIR> <1 if equal>".
template <typename C, int L, int DIR>
static void half_check(const char* name) {
  constexpr int TT = L / 8;
  constexpr int M = log2i(L);
  constexpr int R0 = (M % 3 == 1) ? 2 : (M % 3 == 2) ? 4 : 8;
  const std::vector<C> tw = twiddles<C>();
  unsigned long long seed = 0x2545F4914F6CDD1DULL ^ (unsigned long long)(L * 17 + (DIR > 0));
  bool ok = true;
  for (int t = 0; t < TT; ++t) {
    C a[8], b[8];
    int da[8], db[8];
    for (int s = 0; s < 8; ++s) {
      const double x = s < 4 ? lcg_unit(seed) : 0.0, y = s < 4 ? lcg_unit(seed) : 0.0;
      a[s].x = (decltype(C::x))x;
      a[s].y = (decltype(C::x))y;
      b[s] = a[s];
    }
    rf_pass<C, L, R0, DIR>(a, t, 1, tw.data(), kTwiddleN / L, da);
    rf_pass_half<C, L, R0, DIR>(b, t, db);
    for (int s = 0; s < 8; ++s) {
      ok &= da[s] == db[s];
      ok &= to_ld(a[s].x) == to_ld(b[s].x) && to_ld(a[s].y) == to_ld(b[s].y);
    }
  }
  std::printf("half %s %d %d %d\n", name, L, DIR, ok ? 1 : 0);
}

template <typename C>
static void half_all(const char* name) {
  half_check<C, 8, -1>(name);
  half_check<C, 16, -1>(name);
  half_check<C, 32, -1>(name);
  half_check<C, 64, -1>(name);
  half_check<C, 128, -1>(name);
  half_check<C, 256, -1>(name);
  half_check<C, 512, -1>(name);
  half_check<C, 1024, -1>(name);
  half_check<C, 2048, -1>(name);
  half_check<C, 128, +1>(name);
  half_check<C, 256, +1>(name);
  half_check<C, 512, +1>(name);
}

// FP32 operations of one whole double-float transform of length L in the
// kernels' schedule (first pass -- in its half-input form when HALF, the
// inputs of slots s >= 4 then zero -- and the rolled radix-8 passes; the
// exchanges move data only).  Prints "ops <L> <DIR> <HALF> <count>".
template <int L, int DIR, bool HALF>
static void count_ops() {
  using C = dcplx;
  constexpr int W = 8, TT = L / 8, M = log2i(L);
  constexpr int R0 = (M % 3 == 0) ? 8 : (1 << (M % 3));
  constexpr int NPASS = (M % 3 == 0) ? M / 3 : M / 3 + 1;
  const std::vector<C> tw = twiddles<C>();
  unsigned long long seed = 0xD1B54A32D192ED03ULL ^ (unsigned long long)L;
  std::vector<C> v(L);
  for (int i = 0; i < L; ++i) {
    const bool zero = HALF && i / TT >= 4;
    v[(i % TT) * W + i / TT].x = dfloat(zero ? 0.0 : lcg_unit(seed));
    v[(i % TT) * W + i / TT].y = dfloat(zero ? 0.0 : lcg_unit(seed));
  }
  std::vector<int> dst(L);
  llg_host_fp32_ops = 0;
  int Ns = 1;
  for (int p = 0; p < NPASS; ++p) {
    if (p > 0) {
      std::vector<C> sm(L);
      for (int i = 0; i < L; ++i) sm[dst[i]] = v[i];
      for (int t = 0; t < TT; ++t)
        for (int s = 0; s < W; ++s) v[t * W + s] = sm[t + TT * s];
      pass<C, L, W, 8, DIR>(v, dst, Ns, tw.data(), nullptr);
      Ns *= 8;
    } else {
      for (int t = 0; t < TT; ++t) {
        if constexpr (HALF) rf_pass_half<C, L, R0, DIR>(&v[t * W], t, &dst[t * W]);
        else rf_pass<C, L, R0, DIR>(&v[t * W], t, 1, tw.data(), kTwiddleN / L, &dst[t * W]);
      }
      Ns *= R0;
    }
  }
  std::printf("ops %d %d %d %llu\n", L, DIR, HALF ? 1 : 0, llg_host_fp32_ops);
}

template <int L>
static void count_all() {
  count_ops<L, -1, false>();
  count_ops<L, -1, true>();
  count_ops<L, +1, false>();
}

int main() {
  count_all<8>();
  count_all<16>();
  count_all<32>();
  count_all<64>();
  count_all<128>();
  count_all<256>();
  count_all<512>();
  count_all<1024>();
  count_all<2048>();
  half_all<float2>("f32");
  half_all<double2>("f64");
  half_all<dcplx>("df");
  all_lengths<float2, 8>("f32");
  all_lengths<double2, 8>("f64");
  all_lengths<float2, 16>("f32");
  all_lengths<double2, 16>("f64");
  all_lengths<dcplx, 8>("df");
  all_lengths<dcplx, 16>("df");
  return 0;
}
