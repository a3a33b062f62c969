// Film column pass with 16 register elements per FFT lane, for column
// lengths whose radix-16 schedule saves a shared-memory exchange (Py = 128,
// 256: one exchange instead of two; 1024: two instead of three).  Same work
// and same tile as the 8-element kernel (1024/Py columns, 3 components), in
// 192-thread blocks: a (component, column) group is Py/16 lanes.
//   load the tile -> forward FFT_y (rows >= ny are zero padding) -> product
//   with the 2D tensor (xx, yy, zz, xy; packed DC/Nyquist column separated
//   by Hermitian symmetry) -> inverse FFT_y -> store rows < ny.
// The tensor records of the tile go to shared memory by bulk copy at entry.
#pragma once

#include "kernels_impl.cuh"

namespace llg {

constexpr int kCol16Threads = 192;

template <typename T, int L>
__device__ __forceinline__ void cols16_body(const ColArgs<T>& a, const DevInst& I, const ColTile& tile,
                                            cplx<T>* smem, uint64_t* bar) {
  using C = cplx<T>;
  constexpr int TT = L / 16;
  constexpr int NC = 1024 / L;                     // columns per block
  constexpr int GSC = rf_padded_len(L) + 1;        // group stride
  static_assert(3 * NC * TT == kCol16Threads, "one group per (component, column)");
  const int tid = threadIdx.x;
  const int t = tid % TT, grp_id = tid / TT;       // group = (component, column)
  const int c = grp_id / NC, col = grp_id % NC;
  const int ncols = tile.ncols;
  const bool active = col < ncols;
  const int kx = tile.kx0 + (active ? col : 0);
  const int Lx = I.Lx, ny = I.ny;
  C* grp = smem + grp_id * GSC;
  C* tw1 = smem + kExch;
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
  for (int e = tid; e < ny * 3 * NC; e += kCol16Threads) {
    const int y = e / (3 * NC), r = e - y * (3 * NC);
    const int cc = r / NC, cl = r % NC;
    if (cl < ncols) smem[(cc * NC + cl) * GSC + rf_pad(y)] = spec[((long long)y * 3 + cc) * Lx + cl];
  }
  __syncthreads();
  C v[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int y = t + TT * s;
    // rows y >= ny <= L/2 are the zero padding: s >= 8 is zero at compile time
    v[s] = (s < 8 && active && y < ny) ? grp[rf_pad(y)] : mk<C>((T)0, (T)0);
  }
  gs();
  regfft16<C, L, -1>(v, grp, t, tw1, 1, gs);
#pragma unroll
  for (int s = 0; s < 16; ++s) grp[rf_pad(t + TT * s)] = v[s];
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
        const C other = smem[((1 - c) * NC + col) * GSC + rf_pad(ky)];   // the other in-plane component
        const T diag = (c == 0) ? n[0] : n[1];
        v[s] = mk<C>(diag * v[s].x + nxy * other.x, diag * v[s].y + nxy * other.y);
      }
    } else {
      T nd[4], nq[4];
      load_tensor_smem(stab, kyf, nd);
      load_tensor_smem(stab, NC * nky + kyf, nq);
      const int km = (L - ky) & (L - 1);
      const T p = (T)0.5 * (nd[c] + nq[c]), q = (T)0.5 * (nd[c] - nq[c]);
      const C vb = cconj(grp[rf_pad(km)]);
      v[s] = cadd(cscale(v[s], p), cscale(vb, q));
    }
  }
  __syncthreads();
  regfft16<C, L, 1>(v, grp, t, tw1, 1, gs);
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int y = t + TT * s;
    if (s < 8 && y < ny) grp[rf_pad(y)] = v[s];   // only rows y < ny <= L/2 go back
  }
  __syncthreads();
  for (int e = tid; e < ny * 3 * NC; e += kCol16Threads) {
    const int y = e / (3 * NC), r = e - y * (3 * NC);
    const int cc = r / NC, cl = r % NC;
    if (cl < ncols) spec[((long long)y * 3 + cc) * Lx + cl] = smem[(cc * NC + cl) * GSC + rf_pad(y)];
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
