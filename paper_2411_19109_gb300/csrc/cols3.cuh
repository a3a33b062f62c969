// Column pass of the demag convolution on a 3D grid (nz > 1 layers).
//
// The row kernels leave, for every layer z and row y, the packed half
// spectrum of the x-transform of M = Ms psi m (complex columns kx = 0 ..
// Lx-1, the Nyquist column packed into kx = 0).  For each column kx of its
// tile a block
//   1. transforms the 3 nz (component, layer) sequences along y (zero-padded
//      to Py, register FFTs, several sequences at a time),
//   2. for every ky takes the DFT over the layers (zero-padded to Pz),
//      multiplies by the symmetric 3x3 tensor spectrum N(kx, ky, kz) of the
//      6 components xx, yy, zz, xy, xz, yz at every kz, and transforms back
//      to the layers (unnormalised: -mu0/(Px Py Pz) is in the table),
//   3. transforms every sequence back along y and stores rows y < ny.
// The packed column kx = 0 holds the DC column D and the Nyquist column Q of
// each layer as D + iQ.  Both are real in y for every layer, so their y
// spectra are Hermitian and separate by D(ky) = (Z(ky) + conj Z(-ky))/2,
// Q(ky) = (Z(ky) - conj Z(-ky))/(2i); each goes through step 2 with the
// tensor at kx = 0 resp. kx = Px/2, and the results repack as HD + i HQ.
// One thread owns the pair (ky, -ky) of that column, so a pair's reads and
// writes stay within one thread.
#pragma once

#include "kernels_impl.cuh"

namespace llg {

// 6 tensor components of one (kz, kx, ky) record of the 3D table.
__device__ __forceinline__ void load_tensor6(const float* tab, long long rec, float n[6]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(tab) + 2 * rec);
  const float4 b = __ldg(reinterpret_cast<const float4*>(tab) + 2 * rec + 1);
  n[0] = a.x; n[1] = a.y; n[2] = a.z; n[3] = a.w; n[4] = b.x; n[5] = b.y;
}
__device__ __forceinline__ void load_tensor6(const double* tab, long long rec, double n[6]) {
  const double2* p = reinterpret_cast<const double2*>(tab) + 4 * rec;
  const double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
  n[0] = a.x; n[1] = a.y; n[2] = b.x; n[3] = b.y; n[4] = c.x; n[5] = c.y;
}

// Step 2 for one (kx, ky): out[c][z] = sum_kz W^{-z kz} (N(kx,ky,kz) Mhat)[c],
// Mhat[c](kz) = sum_z M[c][z] W^{z kz}, W = exp(-2 pi i / PZ).  M[c][z] is
// read from shared memory at src + c cstr + z zstr (part 0: the complex
// value, 1: its real part only, 2: its imaginary part only); rec0 is the
// table record of (kz = 0, kx, |ky|), kzrec the record stride between kz
// planes; sy = -1 when ky is a mirrored (negative) frequency.
template <typename T, int PZ>
__device__ __forceinline__ void zconv(const cplx<T>* src, int cstr, int zstr, int part, cplx<T> (&out)[3][PZ / 2],
                                      int nz, const cplx<T>* __restrict__ wz, const T* __restrict__ tab,
                                      long long rec0, long long kzrec, T sy) {
  using C = cplx<T>;
  constexpr int NZM = PZ / 2;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int z = 0; z < NZM; ++z) out[c][z] = mk<C>((T)0, (T)0);
#pragma unroll 1
  for (int kz = 0; kz < PZ; ++kz) {
    C mh[3] = {mk<C>((T)0, (T)0), mk<C>((T)0, (T)0), mk<C>((T)0, (T)0)};
#pragma unroll
    for (int z = 0; z < NZM; ++z) {
      if (z >= nz) break;
      const C w = wz[(z * kz) & (PZ - 1)];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C m = src[c * cstr + z * zstr];
        if (part == 1) m.y = (T)0;
        else if (part == 2) m = mk<C>(m.y, (T)0);
        mh[c] = cadd(mh[c], cmul(m, w));
      }
    }
    const bool lo = kz <= PZ / 2;
    const T sz = lo ? (T)1 : (T)-1;
    T n[6];
    load_tensor6(tab, rec0 + (long long)(lo ? kz : PZ - kz) * kzrec, n);
    const T nxy = sy * n[3], nxz = sz * n[4], nyz = sy * sz * n[5];
    C h[3];
    h[0] = cadd(cadd(cscale(mh[0], n[0]), cscale(mh[1], nxy)), cscale(mh[2], nxz));
    h[1] = cadd(cadd(cscale(mh[0], nxy), cscale(mh[1], n[1])), cscale(mh[2], nyz));
    h[2] = cadd(cadd(cscale(mh[0], nxz), cscale(mh[1], nyz)), cscale(mh[2], n[2]));
#pragma unroll
    for (int z = 0; z < NZM; ++z) {
      if (z >= nz) break;
      const C w = cconj(wz[(z * kz) & (PZ - 1)]);
#pragma unroll
      for (int c = 0; c < 3; ++c) out[c][z] = cadd(out[c][z], cmul(h[c], w));
    }
  }
}

template <typename T, int L, int PZ>
__device__ __forceinline__ void cols3_body(const ColArgs<T>& a, const DevInst& I, const ColTile& tile,
                                           cplx<T>* smem) {
  using C = cplx<T>;
  constexpr int TT = L / 8;
  constexpr int NG = kColThreads / TT;             // FFT groups working at once
  constexpr int GSC = rf_padded_len(L) + 1;
  constexpr int NZM = PZ / 2;
  const int tid = threadIdx.x;
  const int nz = I.nz, ny = I.ny, Lx = I.Lx;
  const int ncols = tile.ncols;
  const int nseq = 3 * nz * ncols;                 // sequence (c, z, col) at ((c nz + z) ncols + col) GSC
  C* tw1 = smem + (long long)nseq * GSC;
  C* wz = tw1 + L;
  C* spec = a.spec + I.spec_off + tile.kx0;
  load_twiddles(tw1, a.tw, L);
  for (int k = tid; k < PZ; k += kColThreads) wz[k] = a.tw[k * (kTwiddleN / PZ)];
  // coalesced load: global rows (z, y), then components, columns fastest
  for (int e = tid; e < nz * ny * 3 * ncols; e += kColThreads) {
    const int col = e % ncols;
    const int r3 = e / ncols;
    const int c = r3 % 3, r = r3 / 3;             // r = z ny + y
    const int y = r % ny, z = r / ny;
    smem[((c * nz + z) * ncols + col) * GSC + rf_pad(y)] = spec[((long long)r * 3 + c) * Lx + col];
  }
  __syncthreads();
  const int t = tid % TT, gid = tid / TT;
  const GroupSync gs = group_sync(TT);
  // 1. forward FFTs along y
  for (int q0 = 0; q0 < nseq; q0 += NG) {
    const int q = q0 + gid;
    if (q < nseq) {
      C* grp = smem + (long long)q * GSC;
      C v[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int y = t + TT * s;
        v[s] = (s < 4 && y < ny) ? grp[rf_pad(y)] : mk<C>((T)0, (T)0);   // zero padding: s >= 4
      }
      gs();
      fft1<C, L, -1>(v, grp, 1, t, tw1, 1, gs);
#pragma unroll
      for (int s = 0; s < 8; ++s) grp[rf_pad(t + TT * s)] = v[s];
    }
  }
  __syncthreads();
  // 2. z transform, tensor product, inverse z transform per (kx, ky)
  const T* tab = a.tens + I.tens_off;
  const long long nky = L / 2 + 1, nkx = Lx + 1;
  const long long kzrec = nkx * nky;
  const int cstr = nz * ncols * GSC, zstr = ncols * GSC;
  const bool dc = tile.kx0 == 0;                   // column 0 of this tile is the packed DC/Nyquist column
  // 2a. packed column: split every layer's Z = D + iQ into D(ky) in slot ky and
  // Q(ky) in slot L - ky for 0 < ky < L/2; at ky = 0 and L/2 both are real
  // and stay packed as D + iQ.  One thread per pair (ky, L - ky).
  if (dc) {
    for (int e = tid; e < 3 * nz * (L / 2 - 1); e += kColThreads) {
      const int ky = 1 + e % (L / 2 - 1), cz = e / (L / 2 - 1);
      C* sq = smem + (long long)cz * zstr;        // (c, z) sequence of column 0
      const C zp = sq[rf_pad(ky)], zm = cconj(sq[rf_pad(L - ky)]);
      const C s = cadd(zp, zm), d = csub(zp, zm);
      sq[rf_pad(ky)] = mk<C>((T)0.5 * s.x, (T)0.5 * s.y);             // D(ky)
      sq[rf_pad(L - ky)] = mk<C>((T)0.5 * d.y, (T)-0.5 * d.x);        // Q(ky) = d / (2i)
    }
    __syncthreads();
  }
  for (int e = tid; e < ncols * L; e += kColThreads) {
    const int col = e / L, ky = e % L;
    const int kx = tile.kx0 + col;
    const bool lo = ky <= L / 2;
    const int kyf = lo ? ky : L - ky;
    C out[3][NZM];
    C* base = smem + (long long)col * GSC;
    if (kx != 0) {
      zconv<T, PZ>(base + rf_pad(ky), cstr, zstr, 0, out, nz, wz, tab, (long long)kx * nky + kyf, kzrec,
                   lo ? (T)1 : (T)-1);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZM; ++z)
          if (z < nz) base[c * cstr + z * zstr + rf_pad(ky)] = out[c][z];
    } else if (ky == 0 || ky == L / 2) {
      // D and Q real: HD with the kx = 0 tensor, HQ with the kx = Px/2 one
      C hq[3][NZM];
      zconv<T, PZ>(base + rf_pad(ky), cstr, zstr, 1, out, nz, wz, tab, (long long)ky, kzrec, (T)1);
      zconv<T, PZ>(base + rf_pad(ky), cstr, zstr, 2, hq, nz, wz, tab, (long long)Lx * nky + ky, kzrec, (T)1);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZM; ++z)
          if (z < nz) base[c * cstr + z * zstr + rf_pad(ky)] = mk<C>(out[c][z].x, hq[c][z].x);
    } else if (lo) {
      // D(ky) in slot ky -> HD(ky); Q(ky) in slot L - ky -> HQ(ky)
      zconv<T, PZ>(base + rf_pad(ky), cstr, zstr, 0, out, nz, wz, tab, (long long)ky, kzrec, (T)1);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZM; ++z)
          if (z < nz) base[c * cstr + z * zstr + rf_pad(ky)] = out[c][z];
      zconv<T, PZ>(base + rf_pad(L - ky), cstr, zstr, 0, out, nz, wz, tab, (long long)Lx * nky + ky, kzrec, (T)1);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZM; ++z)
          if (z < nz) base[c * cstr + z * zstr + rf_pad(L - ky)] = out[c][z];
    }
  }
  __syncthreads();
  // 2b. packed column: recombine Zout(ky) = HD + i HQ, Zout(-ky) = conj HD + i conj HQ
  if (dc) {
    for (int e = tid; e < 3 * nz * (L / 2 - 1); e += kColThreads) {
      const int ky = 1 + e % (L / 2 - 1), cz = e / (L / 2 - 1);
      C* sq = smem + (long long)cz * zstr;
      const C hd = sq[rf_pad(ky)], hq = sq[rf_pad(L - ky)];
      sq[rf_pad(ky)] = mk<C>(hd.x - hq.y, hd.y + hq.x);
      sq[rf_pad(L - ky)] = mk<C>(hd.x + hq.y, hq.x - hd.y);
    }
    __syncthreads();
  }
  // 3. inverse FFTs along y; rows y < ny go back
  for (int q0 = 0; q0 < nseq; q0 += NG) {
    const int q = q0 + gid;
    if (q < nseq) {
      C* grp = smem + (long long)q * GSC;
      C v[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) v[s] = grp[rf_pad(t + TT * s)];
      gs();
      fft1<C, L, 1>(v, grp, 1, t, tw1, 1, gs);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int y = t + TT * s;
        if (s < 4 && y < ny) grp[rf_pad(y)] = v[s];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < nz * ny * 3 * ncols; e += kColThreads) {
    const int col = e % ncols;
    const int r3 = e / ncols;
    const int c = r3 % 3, r = r3 / 3;
    const int y = r % ny, z = r / ny;
    spec[((long long)r * 3 + c) * Lx + col] = smem[((c * nz + z) * ncols + col) * GSC + rf_pad(y)];
  }
}

template <typename T, int L>
__device__ __forceinline__ void cols3_pz(const ColArgs<T>& a, const DevInst& I, const ColTile& tile, cplx<T>* sm) {
  switch (I.Pz) {
    case 4: cols3_body<T, L, 4>(a, I, tile, sm); break;
    case 8: cols3_body<T, L, 8>(a, I, tile, sm); break;
    case 16: cols3_body<T, L, 16>(a, I, tile, sm); break;
    default: break;
  }
}

template <typename T>
__global__ void __launch_bounds__(kColThreads) cols3_kernel(ColArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevInst sI;
  const ColTile tile = a.tiles[blockIdx.x];
  load_inst(sI, a.inst + tile.inst);
  __syncthreads();
  C* sm = reinterpret_cast<C*>(smem_raw);
  switch (sI.log2Py) {
    case 3: cols3_pz<T, 8>(a, sI, tile, sm); break;
    case 4: cols3_pz<T, 16>(a, sI, tile, sm); break;
    case 5: cols3_pz<T, 32>(a, sI, tile, sm); break;
    case 6: cols3_pz<T, 64>(a, sI, tile, sm); break;
    case 7: cols3_pz<T, 128>(a, sI, tile, sm); break;
    case 8: cols3_pz<T, 256>(a, sI, tile, sm); break;
    case 9: cols3_pz<T, 512>(a, sI, tile, sm); break;
    case 10: cols3_pz<T, 1024>(a, sI, tile, sm); break;
    default: break;
  }
}

template <typename T>
void launch_cols3(const ColArgs<T>& a, int ntiles, size_t smem, cudaStream_t st) {
  if (ntiles > 0) cols3_kernel<T><<<ntiles, kColThreads, smem, st>>>(a);
}
template <typename T>
void smem_cols3(size_t smem) {
  static size_t cur = 0;
  raise_smem_limit(reinterpret_cast<const void*>(cols3_kernel<T>), &cur, smem);
}

}  // namespace llg
