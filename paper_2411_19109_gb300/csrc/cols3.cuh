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
//
// The frequencies kz and -kz are taken together.  With w_z = W^{z kz} =
// c_z + i s_z, A = sum_z M_z c_z and B = sum_z M_z s_z give Mhat(+-kz) =
// A +- iB.  The table holds N(kz) for 0 <= kz <= PZ/2; N(-kz) differs from it
// only in the sign of the xz and yz components, so N = Ne +- No with No
// those two.  Then h(+-kz) = (Ne A + No iB) +- (Ne iB + No A) =: S +- D, and
// the pair's share of the inverse transform is
//   h(kz) conj(w_z) + h(-kz) w_z = 2 c_z S - 2 i s_z D.
// kz = 0 and kz = PZ/2 have real w_z = +-1 and enter once.  One tensor
// record and one pass over the layers per pair: half the work of taking
// the PZ frequencies one by one.
template <typename T>
__device__ __forceinline__ void tensor_apply(const T n[6], T sy, const cplx<T> (&a)[3], const cplx<T> (&b)[3],
                                             cplx<T> (&h)[3]) {
  // h = Ne a + No b; Ne: xx, yy, zz, sy xy; No: xz, sy yz
  using C = cplx<T>;
  const T nxy = sy * n[3], nxz = n[4], nyz = sy * n[5];
  h[0] = mk<C>(n[0] * a[0].x + nxy * a[1].x + nxz * b[2].x, n[0] * a[0].y + nxy * a[1].y + nxz * b[2].y);
  h[1] = mk<C>(nxy * a[0].x + n[1] * a[1].x + nyz * b[2].x, nxy * a[0].y + n[1] * a[1].y + nyz * b[2].y);
  h[2] = mk<C>(n[2] * a[2].x + nxz * b[0].x + nyz * b[1].x, n[2] * a[2].y + nxz * b[0].y + nyz * b[1].y);
}

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
  for (int kz = 0; kz <= NZM; ++kz) {
    T n[6];
    load_tensor6(tab, rec0 + (long long)kz * kzrec, n);
    C A[3], B[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) A[c] = B[c] = mk<C>((T)0, (T)0);
#pragma unroll
    for (int z = 0; z < NZM; ++z) {
      if (z >= nz) break;
      const C w = wz[(z * kz) & (PZ - 1)];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C m = src[c * cstr + z * zstr];
        if (part == 1) m.y = (T)0;
        else if (part == 2) m = mk<C>(m.y, (T)0);
        A[c] = mk<C>(A[c].x + m.x * w.x, A[c].y + m.y * w.x);
        B[c] = mk<C>(B[c].x + m.x * w.y, B[c].y + m.y * w.y);
      }
    }
    if (kz == 0 || kz == NZM) {
      // w_z = +-1: Mhat = A, h = (Ne + No) A
      C h[3];
      tensor_apply(n, sy, A, A, h);
#pragma unroll
      for (int z = 0; z < NZM; ++z) {
        if (z >= nz) break;
        const T wr = ((z * kz) & (PZ - 1)) ? (T)-1 : (T)1;
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c][z] = mk<C>(out[c][z].x + wr * h[c].x, out[c][z].y + wr * h[c].y);
      }
    } else {
      C iB[3], S[3], D[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) iB[c] = mk<C>(-B[c].y, B[c].x);
      tensor_apply(n, sy, A, iB, S);
      tensor_apply(n, sy, iB, A, D);
#pragma unroll
      for (int z = 0; z < NZM; ++z) {
        if (z >= nz) break;
        const C w = wz[(z * kz) & (PZ - 1)];
        const T c2 = w.x + w.x, s2 = w.y + w.y;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          out[c][z] = mk<C>(out[c][z].x + c2 * S[c].x + s2 * D[c].y, out[c][z].y + c2 * S[c].y - s2 * D[c].x);
      }
    }
  }
}

// Element i of a 3D column sequence sits at row_pad(L, i) (the exchange
// layout of both register FFTs).
template <int L>
struct SeqMap {
  __device__ __forceinline__ int operator()(int i) const { return row_pad(L, i); }
};

template <typename T, int L, int PZ>
__device__ __forceinline__ void cols3_body(const ColArgs<T>& a, const DevInst& I, const ColTile& tile,
                                           cplx<T>* smem) {
  using C = cplx<T>;
  // y transforms: 16 elements per lane at Py = 1024 in FP32 (radix-16
  // passes: two exchanges instead of three, and twice the sequences per
  // round), 8 elsewhere
  constexpr int W = (sizeof(T) == 4 && L == 1024) ? 16 : 8;
  constexpr int TT = L / W;
  constexpr int NG = kColThreads / TT;             // FFT groups working at once
  constexpr int GSC = cols3_stride(L);
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
    smem[((c * nz + z) * ncols + col) * GSC + row_pad(L, y)] = spec[((long long)r * 3 + c) * Lx + col];
  }
  __syncthreads();
  const int t = tid % TT, gid = tid / TT;
  const GroupSync gs = group_sync(TT);
  // 1. forward FFTs along y
  for (int q0 = 0; q0 < nseq; q0 += NG) {
    const int q = q0 + gid;
    if (q < nseq) {
      C* grp = smem + (long long)q * GSC;
      C v[W];
#pragma unroll
      for (int s = 0; s < W; ++s) {
        const int y = t + TT * s;
        v[s] = (s < W / 2 && y < ny) ? grp[row_pad(L, y)] : mk<C>((T)0, (T)0);   // zero padding: s >= W/2
      }
      gs();
      if constexpr (W == 16) regfft16<C, L, -1>(v, grp, t, tw1, 1, nullptr, SeqMap<L>{}, gs);
      else fft1<C, L, -1>(v, grp, 1, t, tw1, 1, gs);
#pragma unroll
      for (int s = 0; s < W; ++s) grp[row_pad(L, t + TT * s)] = v[s];
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
      const C zp = sq[row_pad(L, ky)], zm = cconj(sq[row_pad(L, L - ky)]);
      const C s = cadd(zp, zm), d = csub(zp, zm);
      sq[row_pad(L, ky)] = mk<C>((T)0.5 * s.x, (T)0.5 * s.y);             // D(ky)
      sq[row_pad(L, L - ky)] = mk<C>((T)0.5 * d.y, (T)-0.5 * d.x);        // Q(ky) = d / (2i)
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
      zconv<T, PZ>(base + row_pad(L, ky), cstr, zstr, 0, out, nz, wz, tab, (long long)kx * nky + kyf, kzrec,
                   lo ? (T)1 : (T)-1);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZM; ++z)
          if (z < nz) base[c * cstr + z * zstr + row_pad(L, ky)] = out[c][z];
    } else if (ky == 0 || ky == L / 2) {
      // D and Q real: HD with the kx = 0 tensor, HQ with the kx = Px/2 one
      C hq[3][NZM];
      zconv<T, PZ>(base + row_pad(L, ky), cstr, zstr, 1, out, nz, wz, tab, (long long)ky, kzrec, (T)1);
      zconv<T, PZ>(base + row_pad(L, ky), cstr, zstr, 2, hq, nz, wz, tab, (long long)Lx * nky + ky, kzrec, (T)1);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZM; ++z)
          if (z < nz) base[c * cstr + z * zstr + row_pad(L, ky)] = mk<C>(out[c][z].x, hq[c][z].x);
    } else if (lo) {
      // D(ky) in slot ky -> HD(ky); Q(ky) in slot L - ky -> HQ(ky)
      zconv<T, PZ>(base + row_pad(L, ky), cstr, zstr, 0, out, nz, wz, tab, (long long)ky, kzrec, (T)1);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZM; ++z)
          if (z < nz) base[c * cstr + z * zstr + row_pad(L, ky)] = out[c][z];
      zconv<T, PZ>(base + row_pad(L, L - ky), cstr, zstr, 0, out, nz, wz, tab, (long long)Lx * nky + ky, kzrec, (T)1);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int z = 0; z < NZM; ++z)
          if (z < nz) base[c * cstr + z * zstr + row_pad(L, L - ky)] = out[c][z];
    }
  }
  __syncthreads();
  // 2b. packed column: recombine Zout(ky) = HD + i HQ, Zout(-ky) = conj HD + i conj HQ
  if (dc) {
    for (int e = tid; e < 3 * nz * (L / 2 - 1); e += kColThreads) {
      const int ky = 1 + e % (L / 2 - 1), cz = e / (L / 2 - 1);
      C* sq = smem + (long long)cz * zstr;
      const C hd = sq[row_pad(L, ky)], hq = sq[row_pad(L, L - ky)];
      sq[row_pad(L, ky)] = mk<C>(hd.x - hq.y, hd.y + hq.x);
      sq[row_pad(L, L - ky)] = mk<C>(hd.x + hq.y, hq.x - hd.y);
    }
    __syncthreads();
  }
  // 3. inverse FFTs along y; rows y < ny go back
  for (int q0 = 0; q0 < nseq; q0 += NG) {
    const int q = q0 + gid;
    if (q < nseq) {
      C* grp = smem + (long long)q * GSC;
      C v[W];
#pragma unroll
      for (int s = 0; s < W; ++s) v[s] = grp[row_pad(L, t + TT * s)];
      gs();
      if constexpr (W == 16) regfft16<C, L, 1>(v, grp, t, tw1, 1, nullptr, SeqMap<L>{}, gs);
      else fft1<C, L, 1>(v, grp, 1, t, tw1, 1, gs);
#pragma unroll
      for (int s = 0; s < W; ++s) {
        const int y = t + TT * s;
        if (s < W / 2 && y < ny) grp[row_pad(L, y)] = v[s];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < nz * ny * 3 * ncols; e += kColThreads) {
    const int col = e % ncols;
    const int r3 = e / ncols;
    const int c = r3 % 3, r = r3 / 3;
    const int y = r % ny, z = r / ny;
    spec[((long long)r * 3 + c) * Lx + col] = smem[((c * nz + z) * ncols + col) * GSC + row_pad(L, y)];
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
__global__ void __launch_bounds__(kColThreads, sizeof(T) == 4 ? 2 : 1) cols3_kernel(ColArgs<T> a) {
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
