// Film column pass with 16 register elements per FFT lane, for column
// lengths whose radix-16 schedule saves a shared-memory exchange (Py = 128,
// 256: one exchange instead of two; 1024: two instead of three).  Same work
// and same tile as the 8-element kernel (1024/Py columns, 3 components), in
// 192-thread blocks: a (component, column) group is Py/16 lanes.
//   load the tile -> forward FFT_y (rows >= ny are zero padding) -> product
//   with the 2D tensor (xx, yy, zz, xy; packed DC/Nyquist column separated
//   by Hermitian symmetry) -> inverse FFT_y -> store rows < ny.
// The tensor records of the tile go to shared memory by bulk copy at entry.
//
// Shared-memory layout: element i of group g sits at base(g) + pad(i).  An
// access wavefront serves 16 lanes of 8 bytes, one per bank pair, so every
// access pattern of the kernel -- natural order t + TT*s, the strided writes
// of each radix pass, the row copies to and from global memory -- must reach
// 16 distinct bank pairs (address mod 16 in complex slots) per half-warp:
//   L = 128 (two groups per half-warp): one pad slot per 8, group stride
//     152 = 8 mod 16 (the two groups of a half-warp fall in opposite halves),
//     plus 2 ((g/2) mod 4) + (g/8) mod 2 so that the row copies, where a
//     half-warp spans 16 groups or parts of two rows, stay distinct;
//   L = 256 (one group per half-warp): one pad slot per 16 (natural order and
//     the radix-16 writes 16 t + r both spread over all pairs), group offsets
//     4 (g mod 4) - g/4 mod 16 for the row copies (12 groups per row);
//   L = 1024: one pad slot per 16, stride 1099.
// The length-agnostic padding of the 8-element kernels (one slot per 8, odd
// group stride) left most accesses here two-way conflicted.
#pragma once

#include "kernels_impl.cuh"

namespace llg {

constexpr int kCol16Threads = 192;

template <int L>
struct Col16Map {
  static constexpr int GS = L == 128 ? 152 : L == 256 ? 288 : 1099;   // group stride
  static constexpr int PL = L == 128 ? L + L / 8 : L + L / 16;          // padded length
  __device__ __forceinline__ static int base(int g) {
    return L == 128 ? g * GS + 2 * ((g >> 1) & 3) + ((g >> 3) & 1)
         : L == 256 ? g * GS + ((4 * (g & 3) - (g >> 2)) & 15)
                    : g * GS;
  }
  __host__ __device__ __forceinline__ constexpr int operator()(int i) const {
    return L == 128 ? i + (i >> 3) : i + (i >> 4);
  }
};

template <typename T, int L>
__device__ __forceinline__ void cols16_body(const ColArgs<T>& a, const DevInst& I, const ColTile& tile,
                                            cplx<T>* smem, uint64_t* bar) {
  using C = cplx<T>;
  constexpr int TT = L / 16;
  constexpr int NC = 1024 / L;                     // columns per block
  using Map = Col16Map<L>;
  constexpr int GSC = Map::GS;
  static_assert(3 * NC * TT == kCol16Threads, "one group per (component, column)");
  static_assert(3 * NC * GSC + L / 16 <= kExch, "groups and the W^4k table fit the exchange area");
  static_assert(Map::PL + (L == 128 ? 7 : L == 256 ? 15 : 0) <= GSC,
                "a group's padded sequence and its offset fit the stride");
  const int tid = threadIdx.x;
  const int t = tid % TT, grp_id = tid / TT;       // group = (component, column)
  const int c = grp_id / NC, col = grp_id % NC;
  const int ncols = tile.ncols;
  const bool active = col < ncols;
  const int kx = tile.kx0 + (active ? col : 0);
  const int Lx = I.Lx, ny = I.ny;
  C* grp = smem + Map::base(grp_id);
  const Map map;
  C* tw1 = smem + kExch;
  C* tw4 = smem + 3 * NC * GSC;                    // W_L^{4k}, k < L/16
  C* spec = a.spec + I.spec_off + tile.kx0;
  const GroupSync gs = group_sync(TT);
  constexpr int nky = L / 2 + 1;
  T* stab = reinterpret_cast<T*>(tw1 + L);
  const T* tab = a.tens + I.tens_off;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
    const unsigned rb = (unsigned)(ncols * nky * 4 * sizeof(T));
    const unsigned nb = tile.kx0 == 0 ? (unsigned)(nky * 4 * sizeof(T)) : 0u;
    mbar_arrive_expect(bar, rb + nb);
    bulk_load(stab, tab + (long long)tile.kx0 * nky * 4, rb, bar);
    if (nb) bulk_load(stab + NC * nky * 4, tab + (long long)Lx * nky * 4, nb, bar);
  }
  load_twiddles(tw1, a.tw, L);
  for (int k = tid; k < L / 16; k += kCol16Threads) tw4[k] = a.tw[k * 4 * (kTwiddleN / L)];
  for (int e = tid; e < ny * 3 * NC; e += kCol16Threads) {
    const int y = e / (3 * NC), r = e - y * (3 * NC);
    const int cc = r / NC, cl = r % NC;
    if (cl < ncols) smem[Map::base(cc * NC + cl) + map(y)] = spec[((long long)y * 3 + cc) * Lx + cl];
  }
  __syncthreads();
  C v[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int y = t + TT * s;
    // rows y >= ny <= L/2 are the zero padding: s >= 8 is zero at compile time
    v[s] = (s < 8 && active && y < ny) ? grp[map(y)] : mk<C>((T)0, (T)0);
  }
  gs();
  regfft16<C, L, -1>(v, grp, t, tw1, 1, tw4, map, gs);
#pragma unroll
  for (int s = 0; s < 16; ++s) grp[map(t + TT * s)] = v[s];
  __syncthreads();
  mbar_wait(bar, 0, a.err);
  const int cl = active ? col : 0;
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int ky = t + TT * s;
    const bool lo = ky <= L / 2;
    const int kyf = lo ? ky : L - ky;
    if (kx != 0) {
      T n[4];
      load_tensor_smem(stab, cl * nky + kyf, n);
      const T nxy = lo ? n[3] : -n[3];
      if (c == 2) {
        v[s] = cscale(v[s], n[2]);
      } else {
        const int go = (1 - c) * NC + col;                              // the other in-plane component
        const C other = smem[Map::base(go) + map(ky)];
        const T diag = (c == 0) ? n[0] : n[1];
        v[s] = mk<C>(diag * v[s].x + nxy * other.x, diag * v[s].y + nxy * other.y);
      }
    } else {
      T nd[4], nq[4];
      load_tensor_smem(stab, kyf, nd);
      load_tensor_smem(stab, NC * nky + kyf, nq);
      const int km = (L - ky) & (L - 1);
      const T p = (T)0.5 * (nd[c] + nq[c]), q = (T)0.5 * (nd[c] - nq[c]);
      const C vb = cconj(grp[map(km)]);
      v[s] = cadd(cscale(v[s], p), cscale(vb, q));
    }
  }
  __syncthreads();
  regfft16<C, L, 1>(v, grp, t, tw1, 1, tw4, map, gs);
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int y = t + TT * s;
    if (s < 8 && y < ny) grp[map(y)] = v[s];   // only rows y < ny <= L/2 go back
  }
  __syncthreads();
  for (int e = tid; e < ny * 3 * NC; e += kCol16Threads) {
    const int y = e / (3 * NC), r = e - y * (3 * NC);
    const int cc = r / NC, cl = r % NC;
    if (cl < ncols) spec[((long long)y * 3 + cc) * Lx + cl] = smem[Map::base(cc * NC + cl) + map(y)];
  }
}

template <typename T>
__global__ void __launch_bounds__(kCol16Threads, sizeof(T) == 4 ? 4 : 1) cols16_kernel(ColArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevInst sI;
  __shared__ uint64_t bar;
  const ColTile tile = a.tiles[blockIdx.x];
  load_inst(sI, a.inst + tile.inst);
  __syncthreads();
  C* sm = reinterpret_cast<C*>(smem_raw);
  switch (sI.log2Py) {
    case 7: cols16_body<T, 128>(a, sI, tile, sm, &bar); break;
    case 8: cols16_body<T, 256>(a, sI, tile, sm, &bar); break;
    case 10: cols16_body<T, 1024>(a, sI, tile, sm, &bar); break;
    default: break;
  }
}

template <typename T>
void launch_cols16(const ColArgs<T>& a, int ntiles, size_t smem, cudaStream_t st) {
  if (ntiles > 0) cols16_kernel<T><<<ntiles, kCol16Threads, smem, st>>>(a);
}
template <typename T>
void smem_cols16(size_t smem) {
  static size_t cur = 0;
  raise_smem_limit(reinterpret_cast<const void*>(cols16_kernel<T>), &cur, smem);
}

}  // namespace llg
