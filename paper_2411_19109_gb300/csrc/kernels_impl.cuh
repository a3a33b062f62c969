// Hot-path kernels of the LLG forward pass and its discrete adjoint.
//
// One RK4 stage is two launches over every instance of the batch:
//   cols_kernel  column pass of the demag convolution: forward FFT along y
//                of the zero-padded row spectra, the pointwise product with
//                the tensor spectrum, inverse FFT along y (register FFTs);
//   rows_kernel  inverse row FFT -> B_d, exchange stencil, anisotropy,
//                Zeeman, LL right-hand side (Eq. 11), RK4 stage combine, and
//                the forward row FFT of the next stage's M = Ms psi Y, all
//                fused per row tile.
// The adjoint stage (adj_kernel) has the same shape: the column pass applies
// the (self-transposed) demag convolution to the field cotangent Bbar.
//
// Spectrum layout per instance: [y][component][kx], Lx = Px/2 complex values
// per row in the packed real-FFT format (element 0 holds the DC and Nyquist
// values as real and imaginary part).  Node arrays: [component][y][x].
#pragma once
#include <climits>

#include "kernels.cuh"
#include "regfft.cuh"
#include "dopri.cuh"
#include "tma.cuh"

namespace llg {

constexpr int kRowThreads = 384;   // 3 components x L/8 lanes x 1024/L rows
constexpr int kColThreads = 384;   // 1024/L columns x 3 components x L/8 lanes
constexpr int kAdjThreads = 384;



// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T edge_weight(T pi, T pj) {
  // w_ij = 2 psi_j/(psi_i + psi_j): harmonic-mean exchange coupling seen by i
  const T s = pi + pj;
  return s > (T)0 ? (T)2 * pj * ((T)1 / s) : (T)0;
}

// Damping a and g = -gamma/(1+a^2) at node (x, y): the interior values, or a
// linear ramp from alpha (W nodes from the edge) to alpha_edge (at the edge)
// inside the absorbing layer.
template <typename T>
__device__ __forceinline__ void damping_at(const DevInst& I, const Coef<T>& K, int x, int y, T& a, T& g) {
  a = K.alpha;
  g = K.gp0;
  if (I.absorb_nodes <= 0) return;
  int d = INT_MAX;
  if (I.absorb_x) d = min(d, min(x, I.nx - 1 - x));
  if (I.absorb_y) d = min(d, min(y, I.ny - 1 - y));
  if (d >= I.absorb_nodes) return;          // ramp (W - d)/W <= 0
  const T ramp = (K.absorb_w - (T)d) * K.inv_absorb_w;
  a = K.alpha + (K.alpha_edge - K.alpha) * ramp;
  g = -(T)kGamma / ((T)1 + a * a);
}

template <typename T>
__device__ __forceinline__ void cross3(const T a[3], const T b[3], T c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T>
__device__ __forceinline__ T dot3(const T a[3], const T b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// LL form of Eq. 11: k = g [Y x B + a Y x (Y x B)], g = -gamma/(1+a^2)
template <typename T>
__device__ __forceinline__ void llg_rhs(const T Y[3], const T B[3], T a, T g, T k[3]) {
  T c1[3], c2[3];
  cross3(Y, B, c1);
  cross3(Y, c1, c2);
  for (int c = 0; c < 3; ++c) k[c] = g * (c1[c] + a * c2[c]);
}

// Cotangents of k = f(Y, B) for a slope cotangent u:
//   Bbar = -g [u x Y + a((u.Y) Y - (Y.Y) u)]
//   mloc = -g [B x u + a((Y.B) u + (u.Y) B - 2 (u.B) Y)]
template <typename T>
__device__ __forceinline__ void rhs_vjp(const T u[3], const T Y[3], const T B[3], T a, T g, T Bbar[3],
                                        T mloc[3]) {
  T uxY[3], Bxu[3];
  cross3(u, Y, uxY);
  cross3(B, u, Bxu);
  const T uY = dot3(u, Y), YY = dot3(Y, Y), YB = dot3(Y, B), uB = dot3(u, B);
  for (int c = 0; c < 3; ++c) {
    Bbar[c] = g * (uxY[c] + a * (uY * Y[c] - YY * u[c]));
    mloc[c] = g * (Bxu[c] + a * (YB * u[c] + uY * B[c] - (T)2 * uB * Y[c]));
  }
}

__device__ __forceinline__ bool in_box(const int b[4], int x, int y) {
  return x >= b[0] && x < b[1] && y >= b[2] && y < b[3];
}

template <typename T>
__device__ __forceinline__ void kahan_add(T& sum, T& comp, T v) {
  const T y = v - comp;
  const T t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

template <typename C>
__device__ __forceinline__ C unpack_one(const C* __restrict__ X, int kk, int L, const C* __restrict__ tw2) {
  // Z[k] = (X_k + conj X_{L-k}) + i W_P^{-k} (X_k - conj X_{L-k}),  P = 2L;  tw2[k] = W_P^k
  const C xk = X[kk];
  if (kk == 0) return mk<C>(xk.x + xk.y, xk.x - xk.y);
  const C xm = cconj(X[L - kk]);
  C w = tw2[kk];
  w.y = -w.y;
  return cadd(cadd(xk, xm), mul_pi(cmul(w, csub(xk, xm))));
}

template <typename C>
__device__ __forceinline__ C pack_one(C zk, C zm_conj, int kk, const C* __restrict__ tw2) {
  // X[k] = (Z_k + conj Z_{L-k})/2 - i W_P^k (Z_k - conj Z_{L-k})/2, X[0] = (Re+Im, Re-Im)
  using R = decltype(C::x);
  if (kk == 0) return mk<C>(zk.x + zk.y, zk.x - zk.y);
  const C w = tw2[kk];
  return cscale(cadd(cadd(zk, zm_conj), mul_mi(cmul(w, csub(zk, zm_conj)))), (R)0.5);
}

// One component's FFT: v[s] holds element t + (L/8)s of the sequence whose
// element i is exchanged through grp[pad(i) * estride].  HALF_IN: v[s] == 0
// for s >= 4 (zero-padded input; see regfft).
template <typename C, int L, int DIR, bool HALF_IN = false>
__device__ __forceinline__ void fft1(C (&v)[8], C* grp, int estride, int t, const C* __restrict__ tw, int tws,
                                     GroupSync sync) {
  regfft<C, L, DIR, 1, HALF_IN>(*reinterpret_cast<C(*)[1][8]>(&v), grp, 0, estride, t, tw, tws, sync);
}

// Row-kernel group stride: the padded length rounded up to even, so that
// every (row slot, component) sequence starts on a 16-byte boundary.
__host__ __device__ constexpr int group_stride(int L) { return (row_padded_len(L) + 1) & ~1; }

// ---------------------------------------------------------------------------
// Thread layout of the row-family kernels (stage, spectrum/field/terminal,
// adjoint): a block of 384 threads covers R = 1024/L rows; thread tid works on
// row slot rl = tid / (3 L/8), field component c = (tid / (L/8)) % 3 and FFT
// lane t = tid % (L/8).  Each (row slot, component) group of L/8 consecutive
// threads owns one padded sequence of the exchange scratch,
// sE + (3 rl + c) * GS, and synchronises only within itself (warp or named
// barrier).  After the inverse FFT the first half of every sequence (complex
// slot j = nodes 2j, 2j+1) is left in natural order; the node phase (all
// threads of the row slot, one node each in turn) reads the field there and
// writes the next FFT's input into the same slots.
// ---------------------------------------------------------------------------

// Twiddles of a row transform: the W_{2L} table tw2 (stride 2), or for the
// double-float transforms the per-pass table that follows it.
template <typename C>
__device__ __forceinline__ const C* row_fft_tw(const C* tw2, int) { return tw2; }
template <>
__device__ __forceinline__ const dcplx* row_fft_tw<dcplx>(const dcplx* tw2, int L) { return tw2 + 2 * L; }

// W_{2L} (and, for double-float, the per-pass table after it) into shared
// memory; the caller synchronises.
template <typename C, int L>
__device__ __forceinline__ void load_row_twiddles(C* tw2, const C* __restrict__ tw4096) {
  load_twiddles(tw2, tw4096, 2 * L);
  if constexpr (RolledPasses<C>::value) fill_pass_twiddles<C, L>(tw2 + 2 * L, tw4096, threadIdx.x, blockDim.x);
}

template <typename T, int L>
__device__ __forceinline__ void row_inverse_comp(cplx<T> (&v)[8], const cplx<T>* __restrict__ X, bool active,
                                                 cplx<T>* grp, int t, const cplx<T>* __restrict__ tw2) {
  using C = cplx<T>;
  constexpr int TT = L / 8;
  const GroupSync gs = group_sync(TT);
#pragma unroll
  for (int s = 0; s < 8; ++s) v[s] = active ? unpack_one(X, t + TT * s, L, tw2) : mk<C>((T)0, (T)0);
  gs();
  fft1<C, L, 1>(v, grp, 1, t, row_fft_tw(tw2, L), 2, gs);
#pragma unroll
  for (int s = 0; s < 4; ++s) grp[seq_pad<C>(L, t + TT * s)] = v[s];
}

// Forward FFT of the node-phase output left in grp (slots j < npairs), packed
// store of the row spectrum component to `out`.
template <typename T, int L>
__device__ __forceinline__ void row_forward_comp(cplx<T>* grp, int npairs, cplx<T>* __restrict__ out, bool active,
                                                 int t, const cplx<T>* __restrict__ tw2) {
  using C = cplx<T>;
  constexpr int TT = L / 8;
  const GroupSync gs = group_sync(TT);
  C v[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int j = t + TT * s;
    v[s] = (s < 4 && j < npairs) ? grp[seq_pad<C>(L, j)] : mk<C>((T)0, (T)0);
  }
  gs();
  fft1<C, L, -1, true>(v, grp, 1, t, row_fft_tw(tw2, L), 2, gs);
#pragma unroll
  for (int s = 0; s < 8; ++s) grp[seq_pad<C>(L, t + TT * s)] = v[s];
  gs();
  if (!active) return;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int kk = t + TT * s;
    const C zm = cconj(grp[seq_pad<C>(L, (L - kk) & (L - 1))]);
    out[kk] = pack_one(v[s], zm, kk, tw2);
  }
}

// Node x of a row slot's three sequences of real type T: complex slot x/2,
// real (x even) or imaginary (x odd) part.
template <typename T, int L>
__device__ __forceinline__ int node_slot(int x) { return 2 * seq_pad<cplx<T>>(L, x >> 1) + (x & 1); }

// ---------------------------------------------------------------------------
// column pass: FFT_y, product with the tensor spectrum, inverse FFT_y.
// Block of 384 threads: 3 components x NC = 1024/L columns groups of L/8
// lanes; group (c, col) owns smem + (c NC + col)(SP + 1) and synchronises
// within itself.  The tile is loaded and stored through shared memory with
// the column index fastest (coalesced); the twiddle table W_L^k, k < L,
// follows the scratch.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void load_tensor(const float* tab, long long idx, float n[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(tab) + idx);
  n[0] = v.x; n[1] = v.y; n[2] = v.z; n[3] = v.w;
}
__device__ __forceinline__ void load_tensor_smem(const float* tab, int idx, float n[4]) {
  const float4 v = reinterpret_cast<const float4*>(tab)[idx];
  n[0] = v.x; n[1] = v.y; n[2] = v.z; n[3] = v.w;
}
__device__ __forceinline__ void load_tensor_smem(const double* tab, int idx, double n[4]) {
  const double2 a = reinterpret_cast<const double2*>(tab)[2 * idx];
  const double2 b = reinterpret_cast<const double2*>(tab)[2 * idx + 1];
  n[0] = a.x; n[1] = a.y; n[2] = b.x; n[3] = b.y;
}
// Record ky of column slot col of a tile's tensor records (nky per column).
// Double-float film tables are planar per column -- the nky hi records
// (xx, yy, zz, xy) then the nky lo records, 16 bytes each -- so that
// consecutive lanes' 16-byte loads meet distinct bank groups (interleaved
// 32-byte records gave every load a 2-way conflict).
template <typename T>
__device__ __forceinline__ void load_tensor_col(const T* tab, int col, int nky, int ky, T n[4]) {
  load_tensor_smem(tab, col * nky + ky, n);
}
template <>
__device__ __forceinline__ void load_tensor_col<dfloat>(const dfloat* tab, int col, int nky, int ky, dfloat n[4]) {
  const float4* q = reinterpret_cast<const float4*>(tab) + 2 * col * nky;
  const float4 h = q[ky], l = q[nky + ky];
  n[0] = dfloat(h.x, l.x); n[1] = dfloat(h.y, l.y); n[2] = dfloat(h.z, l.z); n[3] = dfloat(h.w, l.w);
}
__device__ __forceinline__ void load_tensor(const double* tab, long long idx, double n[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(tab) + 2 * idx);
  const double2 b = __ldg(reinterpret_cast<const double2*>(tab) + 2 * idx + 1);
  n[0] = a.x; n[1] = a.y; n[2] = b.x; n[3] = b.y;
}

template <typename T, int L>
__device__ __forceinline__ void cols_body(const ColArgs<T>& a, const DevInst& I, const ColTile& tile,
                                          cplx<T>* smem, uint64_t* bar) {
  using C = cplx<T>;
  constexpr int TT = L / 8;
  constexpr int NC = 1024 / L;                     // columns per block
  constexpr int GSC = rf_padded_len(L) + 1;        // group stride (odd: spreads banks)
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
  // The tile's tensor records ([col][ky][xx,yy,zz,xy], contiguous in the
  // table) and, for the tile holding kx = 0, those of the Nyquist column go
  // to shared memory by one bulk copy each, behind the load and forward FFT.
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
  if constexpr (RolledPasses<C>::value) fill_pass_twiddles<C, L>(tw1, a.tw, tid, kColThreads);
  else load_twiddles(tw1, a.tw, L);
  // coalesced load of the tile (ny rows x 3 components x NC column slots,
  // columns fastest) into the groups; the divisors are compile-time
  for (int e = tid; e < ny * 3 * NC; e += kColThreads) {
    const int y = e / (3 * NC), r = e - y * (3 * NC);
    const int cc = r / NC, cl = r % NC;
    if (cl < ncols) smem[(cc * NC + cl) * GSC + rf_pad(y)] = spec[((long long)y * 3 + cc) * Lx + cl];
  }
  __syncthreads();
  C v[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int y = t + TT * s;
    // rows y >= ny are the zero padding; ny <= L/2, so s >= 4 is zero
    // at compile time and the first pass folds
    v[s] = (s < 4 && active && y < ny) ? grp[rf_pad(y)] : mk<C>((T)0, (T)0);
  }
  gs();
  fft1<C, L, -1, true>(v, grp, 1, t, tw1, 1, gs);
  // publish every component at every ky for the 3x3 product
#pragma unroll
  for (int s = 0; s < 8; ++s) grp[rf_pad(t + TT * s)] = v[s];
  __syncthreads();
  mbar_wait(bar, 0, a.err);
  const int cl = active ? col : 0;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int ky = t + TT * s;
    const bool lo = ky <= L / 2;
    const int kyf = lo ? ky : L - ky;
    if (kx != 0) {
      T n[4];
      load_tensor_col(stab, cl, nky, kyf, n);
      const T nxy = lo ? n[3] : -n[3];
      if (c == 2) {
        v[s] = cscale(v[s], n[2]);
      } else {
        const C other = smem[((1 - c) * NC + col) * GSC + rf_pad(ky)];   // the other in-plane component
        const T diag = (c == 0) ? n[0] : n[1];
        v[s] = mk<C>(diag * v[s].x + nxy * other.x, diag * v[s].y + nxy * other.y);
      }
    } else {
      // packed DC (kx = 0) and Nyquist (kx = Px/2) columns: separate them by
      // Hermitian symmetry in ky, apply each its own (diagonal) tensor
      T nd[4], nq[4];
      load_tensor_col(stab, 0, nky, kyf, nd);
      load_tensor_col(stab, NC, nky, kyf, nq);
      const int km = (L - ky) & (L - 1);
      const T p = (T)0.5 * (nd[c] + nq[c]), q = (T)0.5 * (nd[c] - nq[c]);
      const C vb = cconj(grp[rf_pad(km)]);
      v[s] = cadd(cscale(v[s], p), cscale(vb, q));
    }
  }
  __syncthreads();
  fft1<C, L, 1>(v, grp, 1, t, tw1, 1, gs);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int y = t + TT * s;
    if (s < 4 && y < ny) grp[rf_pad(y)] = v[s];   // only rows y < ny <= L/2 go back
  }
  __syncthreads();
  for (int e = tid; e < ny * 3 * NC; e += kColThreads) {
    const int y = e / (3 * NC), r = e - y * (3 * NC);
    const int cc = r / NC, cl = r % NC;
    if (cl < ncols) spec[((long long)y * 3 + cc) * Lx + cl] = smem[(cc * NC + cl) * GSC + rf_pad(y)];
  }
}

// MB: the blocks per SM the kernel is compiled for (its register cap):
// FP32 3; FP64 1; double-float 1 or 2 (launch-configuration candidates:
// 32 registers of FFT values per lane make the register cap a trade
// between occupancy and spills).
template <typename T, int MB>
__global__ void __launch_bounds__(kColThreads, MB) cols_kernel(ColArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevInst sI;
  __shared__ uint64_t bar;
  const ColTile tile = a.tiles[blockIdx.x];
  load_inst(sI, a.inst + tile.inst);
  __syncthreads();
  C* sm = reinterpret_cast<C*>(smem_raw);
  switch (sI.log2Py) {
    case 3: cols_body<T, 8>(a, sI, tile, sm, &bar); break;
    case 4: cols_body<T, 16>(a, sI, tile, sm, &bar); break;
    case 5: cols_body<T, 32>(a, sI, tile, sm, &bar); break;
    case 6: cols_body<T, 64>(a, sI, tile, sm, &bar); break;
    case 7: cols_body<T, 128>(a, sI, tile, sm, &bar); break;
    case 8: cols_body<T, 256>(a, sI, tile, sm, &bar); break;
    case 9: cols_body<T, 512>(a, sI, tile, sm, &bar); break;
    case 10: cols_body<T, 1024>(a, sI, tile, sm, &bar); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// staged halo rows
// ---------------------------------------------------------------------------

// Issue the halo copies (rows ylo..yhi-1 of `ncomp` components of F) into a
// staged array with rows y0-1 .. y0+R; returns the bytes issued.
template <typename T>
__device__ __forceinline__ unsigned stage_halo(T* sF, int RM, const T* F, long long nodes, int ncomp, int nx,
                                               int y0, int ylo, int yhi, uint64_t* bar) {
  const unsigned hb = (unsigned)((yhi - ylo) * nx * sizeof(T));
  const int r0 = ylo - y0 + 1;
  for (int c = 0; c < ncomp; ++c)
    bulk_load(sF + (c * (RM + 2) + r0) * nx, F + c * nodes + (long long)ylo * nx, hb, bar);
  return hb * ncomp;
}

// Common per-block geometry of the row-family kernels.
template <int L>
struct RowGeom {
  static constexpr int TT = L / 8;
  static constexpr int SP = row_padded_len(L);
  static constexpr int RM = rows_per_tile(L);
  int rl, c, t, tr;
  __device__ __forceinline__ RowGeom(int tid) {
    t = tid % TT;
    c = (tid / TT) % 3;
    rl = tid / (3 * TT);
    tr = c * TT + t;        // lane within the row (0 .. 3 TT - 1)
  }
};

// ---------------------------------------------------------------------------
// row pass variants run once per segment or call: spectrum of M = Ms psi Y,
// effective field, terminal energies / lambda_N.  Shared memory: scratch
// (kExch complex) then W_{2L}^k, k < 2L.
// ---------------------------------------------------------------------------

template <typename T, int L, int MODE, bool Z3>
__device__ __forceinline__ void rows_body(const RowArgs<T>& a, const DevInst& I, const RowTile& tile,
                                          cplx<T>* smem, double* red, T rf) {
  using C = cplx<T>;
  using G = RowGeom<L>;
  constexpr int GS = group_stride(L);
  const G g(threadIdx.x);
  const bool active = g.rl < tile.nrows;
  const int nx = I.nx, ny = I.ny;
  const int y = tile.y0 + (active ? g.rl : 0);
  const int z = tile.z, nz = I.nz;
  const long long nodes = I.nodes, layer = I.layer;
  const long long zoff = (long long)z * layer;   // first node of the tile's layer
  C* sE = smem + g.rl * 3 * GS;        // the three sequences of this row slot
  C* grp = sE + g.c * GS;
  T* sEr = reinterpret_cast<T*>(sE);
  C* tw2 = smem + kExch;
  C* row = a.spec + I.spec_off + ((long long)z * ny + y) * 3 * L;
  const long long off3 = 3 * I.node_off;
  const T* __restrict__ Y = a.Yin + off3;
  const T* __restrict__ ps = a.psi + I.node_off;
  const Coef<T>& K = coef<T>(I);
  const T Ms = K.Ms, cx = K.cx, cy = K.cy, cz = K.cz, kan = K.kan;
  const T ku[3] = {K.ku[0], K.ku[1], K.ku[2]};
  load_twiddles(tw2, a.tw, 2 * L);
  __syncthreads();
  if (MODE != ROW_FFT_ONLY && MODE != ROW_DP_START) {
    C v[8];
    row_inverse_comp<T, L>(v, row + g.c * L, active, grp, g.t, tw2);
    __syncthreads();
  }
  // Dormand-Prince attempt start: this instance's acceptance of the last
  // attempt (then m <- y5, k_1 <- k_7, m stored at checkpoint slot cnt) and
  // the first stage input Y_2 = m + h a(2, 1) k_1
  const bool dp_acc = MODE == ROW_DP_START && a.accept[tile.inst] != 0;
  const T dp_h = MODE == ROW_DP_START ? (T)a.hst[4 * tile.inst + 1] : (T)0;
  const int dp_every = a.ck_every > 1 ? a.ck_every : 1;
  const long long dp_slot = MODE == ROW_DP_START && a.ckall && a.cnt[tile.inst] % dp_every == 0
                                ? (long long)(a.cnt[tile.inst] / dp_every) * a.kstride
                                : -1;
  double vsum = 0.0;
#pragma unroll 1
  for (int x = g.tr; active && x < nx; x += 3 * G::TT) {
    const long long n0 = zoff + (long long)y * nx + x;
    const int sl = node_slot<T, L>(x);
    if (MODE == ROW_FFT_ONLY) {
      const T p = ps[n0];
#pragma unroll
      for (int c = 0; c < 3; ++c) sEr[2 * c * GS + sl] = Ms * p * Y[c * nodes + n0];
      continue;
    }
    if (MODE == ROW_DP_START) {
      const T p = ps[n0];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long id = off3 + c * nodes + n0;
        T mv, k1;
        if (dp_acc) {
          mv = a.y5[id];
          k1 = a.kbuf[6 * a.kstride + id];
          a.mout[id] = mv;
          a.kbuf[id] = k1;
          if (dp_slot >= 0) a.ckall[dp_slot + id] = mv;
        } else {
          mv = a.m[id];
          k1 = a.kbuf[id];
        }
        // associated as the stage kernel forms Y_{s+1} = m + h (a k), so
        // that a stage recomputed from m (reverse sweep, replay) repeats
        // this one bit for bit
        const T acc2 = a.dpa[0] * k1;
        const T y2 = mv + dp_h * acc2;
        a.Yout[id] = y2;
        sEr[2 * c * GS + sl] = Ms * p * y2;
      }
      continue;
    }
    T Bd[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Bd[c] = sEr[2 * c * GS + sl];
    if (MODE == ROW_FIELD && a.demag_only) {
#pragma unroll
      for (int c = 0; c < 3; ++c) a.Bout[off3 + c * nodes + n0] = Bd[c];
      continue;
    }
    // own value and the neighbours (+x, -x, +y, -y, +z, -z) from global memory
    T yi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) yi[c] = Y[c * nodes + n0];
    const T pi = ps[n0];
    T Bex[3] = {0, 0, 0};
    T qpsi = 0, eex = 0;
    const T hh[6] = {K.ihx2, K.ihx2, K.ihy2, K.ihy2, K.ihz2, K.ihz2};
    const T cc[6] = {cx, cx, cy, cy, cz, cz};
#pragma unroll
    for (int d = 0; d < (Z3 ? 6 : 4); ++d) {
      const bool ok = d == 0 ? x + 1 < nx : d == 1 ? x > 0 : d == 2 ? y + 1 < ny : d == 3 ? y > 0
                    : d == 4 ? z + 1 < nz : z > 0;
      if (!ok) continue;
      const long long j = n0 + (d == 0 ? 1 : d == 1 ? -1 : d == 2 ? nx : d == 3 ? -nx : d == 4 ? layer : -layer);
      const T pj = ps[j];
      const T w = cc[d] * edge_weight(pi, pj);
      T dm2 = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T dd = Y[c * nodes + j] - yi[c];
        Bex[c] += w * dd;
        dm2 += dd * dd;
      }
      if (MODE == ROW_TERMINAL && I.objective == 1) {
        const T sp = pi + pj;
        const T Aij = sp > (T)0 ? (T)2 * K.A * pi * pj / sp : (T)0;
        eex += (T)0.5 * Aij * dm2 * hh[d];
        if (sp > (T)0) qpsi += (T)2 * K.A * pj * pj / (sp * sp) * dm2 * hh[d];
      }
    }
    if (MODE == ROW_TERMINAL) {
      T lam[3] = {0, 0, 0};
      T qp = 0;
      if (I.objective == 1) {
        const T V = K.V, sc = K.escale;
        const T mdb = dot3(yi, Bd);
        vsum += -0.5 * (double)V * (double)Ms * (double)pi * (double)mdb + (double)V * (double)eex;
        qp = qpsi * V * sc - V * Ms * mdb * sc;
        double psum = 0.0;   // the per-tile psi partials, added in tile order
        for (int t = 0; t < I.ntile; ++t) psum += a.psitile[I.tile_off + t];
        const double meanpsi = psum / (double)nodes;
        qp += (T)(2.0 * I.penalty_w * (meanpsi - I.area_target) / (double)nodes);
#pragma unroll
        for (int c = 0; c < 3; ++c) lam[c] = -V * Ms * pi * (Bd[c] + Bex[c]) * sc;
      } else if (I.objective == 2) {
        if (a.nsteps >= a.n_from) {
#pragma unroll
          for (int b = 0; b < 2; ++b)
            if (in_box(I.boxes[b], x, y)) lam[I.comp] += (T)a.wtab[I.wt_off + 2 * a.nsteps + b];
        }
      } else if (I.objective == 3) {
        // a sample at step N: w sign(P - T)/S on lambda_comp (psi-weighted)
        // and the quotient-rule term on dJ/dpsi; then the size and centre
        // terms of Eq. 9, from the per-tile psi moments
        const double wl = a.wtab[I.wt_off + 2 * a.nsteps];
        lam[I.comp] = (T)(wl * (double)pi);
        double q = wl * (double)yi[I.comp] - a.wtab[I.wt_off + 2 * a.nsteps + 1];
        double S = 0.0, Sx = 0.0, Sy = 0.0;
        for (int t = 0; t < I.ntile; ++t) {
          S += a.psitile[I.tile_off + t];
          Sx += a.psimom[2 * (I.tile_off + t)];
          Sy += a.psimom[2 * (I.tile_off + t) + 1];
        }
        const double xc = Sx / S, yc = Sy / S;
        const double sgx = xc > I.centre_x0 ? 1.0 : (xc < I.centre_x0 ? -1.0 : 0.0);
        const double sgy = yc > I.centre_y0 ? 1.0 : (yc < I.centre_y0 ? -1.0 : 0.0);
        q += 2.0 * I.penalty_w * (S / (double)nodes - I.area_target) / (double)nodes;
        q += I.centre_w * (sgx * ((double)x - xc) + sgy * ((double)y - yc)) / S;
        qp = (T)q;
      } else if (a.nsteps >= a.n_from) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          if (!in_box(I.boxes[b], x, y)) continue;
          const T vv = yi[I.comp];
          lam[I.comp] += K.wbox[b] * (I.power == 2 ? (T)2 * vv : (T)1);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) a.lam[off3 + c * nodes + n0] = lam[c];
      a.psib[I.node_off + n0] = qp;
      a.psic[I.node_off + n0] = (T)0;
      continue;
    }
    // ROW_FIELD: full effective field
    T B[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) B[c] = Bd[c] + Bex[c] + K.B_bias[c];
    if (kan != (T)0) {
      const T dd = dot3(yi, ku);
#pragma unroll
      for (int c = 0; c < 3; ++c) B[c] += kan * dd * ku[c];
    }
    if (in_box(I.src, x, y)) {
#pragma unroll
      for (int c = 0; c < 3; ++c) B[c] += rf * K.rf_dir[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) a.Bout[off3 + c * nodes + n0] = B[c];
  }
  if (MODE == ROW_TERMINAL) {
    if (I.objective == 1) {
      const double tot = block_sum(vsum, red);
      if (threadIdx.x == 0) a.jterm[I.tile_off + tile.k] = tot * I.escale;
    }
    return;
  }
  if (MODE == ROW_FIELD) return;
  __syncthreads();
  row_forward_comp<T, L>(grp, nx / 2, row + g.c * L, active, g.t, tw2);
}

// ---------------------------------------------------------------------------
// forward RK4 stage.  At entry one thread issues cp.async.bulk copies of the
// tile's packed field spectrum (barrier 0) and of the halo rows the stencil
// reads, Y_s and psi with one row on each side (barrier 1); the inverse row
// FFTs run while the halo rows, m_n and the RK accumulator (also barrier 1)
// are in flight.  Shared memory: [scratch kExch complex][Y halo 3 x (R+2)
// rows][psi halo (R+2) rows][m 3 x R rows][acc 3 x R rows][W_{2L}^k, k < 2L].
// ---------------------------------------------------------------------------

template <typename T, int L, bool Z3, bool DP>
__device__ __forceinline__ void stage_body(const RowArgs<T>& a, const DevInst& I, const RowTile& tile,
                                           unsigned char* smem_raw, uint64_t* bars, double* red, T rf) {
  using C = cplx<T>;
  using G = RowGeom<L>;
  constexpr int RM = G::RM;
  constexpr int GS = group_stride(L);
  const G g(threadIdx.x);
  const int tid = threadIdx.x;
  const int nr = tile.nrows;
  const bool active = g.rl < nr;
  const int nx = I.nx, ny = I.ny, y0 = tile.y0;
  const int y = y0 + (active ? g.rl : 0);
  const int z = tile.z, nz = I.nz;
  const long long nodes = I.nodes, layer = I.layer;
  const long long zoff = (long long)z * layer;   // first node of the tile's layer
  C* sx = reinterpret_cast<C*>(smem_raw);
  T* sY = reinterpret_cast<T*>(sx + kExch);
  T* sP = sY + 3 * (RM + 2) * nx;
  C* tw2 = reinterpret_cast<C*>(sP + (RM + 2) * nx);
  C* sE = sx + g.rl * 3 * GS;
  C* grp = sE + g.c * GS;
  T* sEr = reinterpret_cast<T*>(sE);
  const long long off3 = 3 * I.node_off;
  C* row0 = a.spec + I.spec_off + ((long long)z * ny + y0) * 3 * L;
  const int s = a.stage;
  const long long n = (a.step_base ? *a.step_base : 0) + a.local_step;
  const int ylo = max(0, y0 - 1), yhi = min(ny, y0 + nr + 1);
  T* __restrict__ gacc = a.acc;
  const T* __restrict__ gm = a.m;
  T* __restrict__ gYout = a.Yout;
  T* __restrict__ gmout = a.mout;
  T* __restrict__ gB = a.Bout;
  T* __restrict__ gck = a.ckpt;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  load_twiddles(tw2, a.tw, 2 * L);
  __syncthreads();
  if (tid == 0) {
    // each (row, component) spectrum lands at the start of its own group
    const unsigned rowb = (unsigned)(L * sizeof(C));
    mbar_arrive_expect(&bars[0], nr * 3 * rowb);
    for (int r = 0; r < nr; ++r)
      for (int c = 0; c < 3; ++c) bulk_load(sx + (r * 3 + c) * GS, row0 + (r * 3 + c) * L, rowb, &bars[0]);
    const unsigned hb = (unsigned)((yhi - ylo) * nx * sizeof(T));
    mbar_arrive_expect(&bars[1], 4 * hb);
    stage_halo(sY, RM, a.Yin + off3 + zoff, nodes, 3, nx, y0, ylo, yhi, &bars[1]);
    stage_halo(sP, RM, a.psi + I.node_off + zoff, nodes, 1, nx, y0, ylo, yhi, &bars[1]);
  }
  mbar_wait(&bars[0], 0, a.err);
  {
    C v[8];
    row_inverse_comp<T, L>(v, grp, active, grp, g.t, tw2);
  }
  mbar_wait(&bars[1], 0, a.err);
  __syncthreads();

  const Coef<T>& K = coef<T>(I);
  const T Ms = K.Ms, cx = K.cx, cy = K.cy, cz = K.cz, kan = K.kan;
  const T ku[3] = {K.ku[0], K.ku[1], K.ku[2]};
  const T dt = (T)a.dt;
  const T hs = (s == 1 || s == 2) ? (T)0.5 * dt : dt;     // Y_{s+1} = m + hs k_s
  const int cs = (RM + 2) * nx;                            // component stride of the staged halo
  double vsum = 0.0;
  // Dormand-Prince: this instance's step size h, the slope slots, and the
  // error sum of stage 7
  const T hdp = DP ? (T)a.hst[4 * tile.inst + 1] : (T)0;
  double esum = 0.0;
  const bool objective_step = !DP && s == 4 && a.slots != nullptr && I.objective == 0 && (n + 1) >= a.n_from;
  // spectral objective: the port-box sums of m_comp at step n + 1; curve
  // objective: the tile's sum of psi m_comp (channel 0) at every step
  const bool spectral_step = !DP && s == 4 && a.pslots != nullptr &&
                             ((I.objective == 2 && (n + 1) >= a.n_from) || I.objective == 3);
  T psum[2] = {0, 0};   // per-thread partials in T (a thread adds a few nodes), tile sum in FP64
#pragma unroll 1
  for (int x = g.tr; active && x < nx; x += 3 * G::TT) {
    const long long n0 = zoff + (long long)y * nx + x;
    const int sl = node_slot<T, L>(x);
    const int oi = (g.rl + 1) * nx + x;
    // m_n and the RK accumulator of this node first (their latencies overlap
    // the field assembly below)
    T mn[3], ac[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = off3 + c * nodes + n0;
      mn[c] = gm[id];
      ac[c] = (!DP && s > 1) ? gacc[id] : (T)0;
    }
    const T pi = sP[oi];
    T yi[3], B[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      yi[c] = sY[c * cs + oi];
      B[c] = sEr[2 * c * GS + sl] + K.B_bias[c];
    }
    // exchange: sum over existing neighbours of c_d w_ij (Y_j - Y_i)
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const bool ok = d == 0 ? x + 1 < nx : d == 1 ? x > 0 : d == 2 ? y + 1 < ny : y > 0;
      if (!ok) continue;
      const int oj = oi + (d == 0 ? 1 : d == 1 ? -1 : d == 2 ? nx : -nx);
      const T w = (d < 2 ? cx : cy) * edge_weight(pi, sP[oj]);
#pragma unroll
      for (int c = 0; c < 3; ++c) B[c] += w * (sY[c * cs + oj] - yi[c]);
    }
    // the layers above and below (3D), from global memory
    if constexpr (Z3) {
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        if (d == 0 ? z + 1 >= nz : z == 0) continue;
        const long long j = n0 + (d == 0 ? layer : -layer);
        const T w = cz * edge_weight(pi, a.psi[I.node_off + j]);
#pragma unroll
        for (int c = 0; c < 3; ++c) B[c] += w * (a.Yin[off3 + c * nodes + j] - yi[c]);
      }
    }
    if (kan != (T)0) {
      const T dd = dot3(yi, ku);
#pragma unroll
      for (int c = 0; c < 3; ++c) B[c] += kan * dd * ku[c];
    }
    if (in_box(I.src, x, y)) {
#pragma unroll
      for (int c = 0; c < 3; ++c) B[c] += rf * K.rf_dir[c];
    }
    T k[3], al, ga;
    damping_at(I, K, x, y, al, ga);
    llg_rhs(yi, B, al, ga, k);
    if constexpr (DP) {
      // k_s into its slot; then Y_{s+1} = m + h sum_{j<=s} a(s+1, j) k_j, or
      // at stage 7 (Y_7 = y5) the error h sum_j e_j k_j scaled per node and
      // component by atol + rtol max(|psi m|, |psi y5|), measured on psi e
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long id = off3 + c * nodes + n0;
        if (gB) gB[id] = B[c];
        a.kbuf[(long long)(s - 1) * a.kstride + id] = k[c];
        if (s < 7) {
          T acc2 = a.dpa[s - 1] * k[c];
          // fully unrolled: the slot loads of all earlier stages issue together
#pragma unroll
          for (int j = 1; j < 6; ++j)
            if (j < s && a.dpa[j - 1] != (T)0) acc2 += a.dpa[j - 1] * a.kbuf[(long long)(j - 1) * a.kstride + id];
          const T yv = mn[c] + hdp * acc2;
          gYout[id] = yv;
          sEr[2 * c * GS + sl] = Ms * pi * yv;
        } else {
          T ec = a.dpe[6] * k[c];
#pragma unroll
          for (int j = 1; j < 7; ++j)
            if (a.dpe[j - 1] != (T)0) ec += a.dpe[j - 1] * a.kbuf[(long long)(j - 1) * a.kstride + id];
          const double p = (double)pi;
          const double sc = a.atol + a.rtol * fmax(fabs(p * (double)mn[c]), fabs(p * (double)yi[c]));
          const double r = p * (double)hdp * (double)ec / sc;
          esum += r * r;
        }
      }
      continue;
    }
    T yn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = off3 + c * nodes + n0;
      if (gB) gB[id] = B[c];
      const T m0 = mn[c];
      if (s == 1) {
        gacc[id] = k[c];
        yn[c] = m0 + hs * k[c];
      } else if (s < 4) {
        gacc[id] = ac[c] + (T)2 * k[c];
        yn[c] = m0 + hs * k[c];
      } else {
        yn[c] = m0 + dt / (T)6 * (ac[c] + k[c]);
        gmout[id] = yn[c];
        if (gck) gck[id] = yn[c];
      }
      if (s < 4) gYout[id] = yn[c];
      sEr[2 * c * GS + sl] = Ms * pi * yn[c];
    }
    if (objective_step) {
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        if (!in_box(I.boxes[b], x, y)) continue;
        const T vv = yn[I.comp];
        vsum += I.wbox[b] * (double)(I.power == 2 ? vv * vv : vv);
      }
    }
    if (spectral_step) {
      if (I.objective == 3) {
        psum[0] += pi * yn[I.comp];
      } else {
#pragma unroll
        for (int b = 0; b < 2; ++b)
          if (in_box(I.boxes[b], x, y)) psum[b] += yn[I.comp];
      }
    }
  }
  if (objective_step) {
    bool touches = false;
    for (int b = 0; b < 2; ++b)
      touches |= (I.wbox[b] != 0.0) && I.boxes[b][2] < y0 + nr && I.boxes[b][3] > y0;
    if (touches) {
      const double tot = block_sum(vsum, red);
      if (threadIdx.x == 0) a.slots[I.slot_off + (long long)(n + 1) * I.ntile + tile.k] = tot;
    }
  }
  if (DP && s == 7) {
    const double tot = block_sum(esum, red);
    if (threadIdx.x == 0) a.eslots[I.tile_off + tile.k] = tot;
    return;   // no next stage: no spectrum to form
  }
  if (spectral_step) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (I.objective == 3 ? b != 0
                           : !(I.boxes[b][2] < y0 + nr && I.boxes[b][3] > y0 && I.boxes[b][0] < I.boxes[b][1]))
        continue;
      const double tot = block_sum((double)psum[b], red);
      if (threadIdx.x == 0) a.pslots[2 * (I.slot_off + (long long)(n + 1) * I.ntile + tile.k) + b] = tot;
      __syncthreads();   // red is reused by the next box
    }
  }
  __syncthreads();
  row_forward_comp<T, L>(grp, nx / 2, a.spec + I.spec_off + ((long long)z * ny + y) * 3 * L + g.c * L, active, g.t,
                         tw2);
}

// Stage body for the row FFT length of the tile's instance; Z3 selects the
// 3D variant (z neighbours), so film tiles carry none of its registers.
template <typename T, bool Z3, bool DP>
__device__ __forceinline__ void stage_dispatch(const RowArgs<T>& a, const DevInst& I, const RowTile& tile,
                                               unsigned char* smem_raw, uint64_t* bars, double* red, T rf) {
  switch (I.log2Lx) {
    case 3: stage_body<T, 8, Z3, DP>(a, I, tile, smem_raw, bars, red, rf); break;
    case 4: stage_body<T, 16, Z3, DP>(a, I, tile, smem_raw, bars, red, rf); break;
    case 5: stage_body<T, 32, Z3, DP>(a, I, tile, smem_raw, bars, red, rf); break;
    case 6: stage_body<T, 64, Z3, DP>(a, I, tile, smem_raw, bars, red, rf); break;
    case 7: stage_body<T, 128, Z3, DP>(a, I, tile, smem_raw, bars, red, rf); break;
    case 8: stage_body<T, 256, Z3, DP>(a, I, tile, smem_raw, bars, red, rf); break;
    case 9: stage_body<T, 512, Z3, DP>(a, I, tile, smem_raw, bars, red, rf); break;
    case 10: stage_body<T, 1024, Z3, DP>(a, I, tile, smem_raw, bars, red, rf); break;
    default: break;
  }
}

// Z3: the 3D variant (z neighbours); film tiles launch the variant without
// them, which needs fewer registers.
template <typename T, int MODE, bool Z3>
__global__ void __launch_bounds__(kRowThreads, sizeof(T) == 4 ? ((Z3 || MODE >= ROW_DP_STAGE) ? 2 : 3) : 1)
    rows_kernel(RowArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kRowThreads / 32];
  __shared__ DevInst sI;
  __shared__ double s_rf;
  __shared__ uint64_t bars[2];
  const RowTile tile = a.tiles[blockIdx.x];
  load_inst(sI, a.inst + tile.inst);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (MODE == ROW_FIELD) {
      s_rf = sI.b_rf * sin(2.0 * M_PI * sI.f_rf * a.t_field);
    } else if (MODE == ROW_STAGE) {
      const long long n = (a.step_base ? *a.step_base : 0) + a.local_step;
      const int c = (a.stage == 1) ? 0 : (a.stage == 4 ? 2 : 1);
      s_rf = a.rf[sI.rf_off + 3 * n + c];
    } else if (MODE == ROW_DP_STAGE) {
      // the sine drive at the stage time t + c_s h of this instance's attempt
      const double t0 = a.hst[4 * tile.inst], h = a.hst[4 * tile.inst + 1];
      s_rf = sI.b_rf * sin(2.0 * M_PI * sI.f_rf * (t0 + dp::c(a.stage) * h));
    } else {
      s_rf = 0.0;
    }
  }
  __syncthreads();
  C* sm = reinterpret_cast<C*>(smem_raw);
  const T rf = (T)s_rf;
  if (MODE == ROW_STAGE || MODE == ROW_DP_STAGE) {
    stage_dispatch<T, Z3, MODE == ROW_DP_STAGE>(a, sI, tile, smem_raw, bars, red, rf);
    return;
  }
  switch (sI.log2Lx) {
    case 3: rows_body<T, 8, MODE, Z3>(a, sI, tile, sm, red, rf); break;
    case 4: rows_body<T, 16, MODE, Z3>(a, sI, tile, sm, red, rf); break;
    case 5: rows_body<T, 32, MODE, Z3>(a, sI, tile, sm, red, rf); break;
    case 6: rows_body<T, 64, MODE, Z3>(a, sI, tile, sm, red, rf); break;
    case 7: rows_body<T, 128, MODE, Z3>(a, sI, tile, sm, red, rf); break;
    case 8: rows_body<T, 256, MODE, Z3>(a, sI, tile, sm, red, rf); break;
    case 9: rows_body<T, 512, MODE, Z3>(a, sI, tile, sm, red, rf); break;
    case 10: rows_body<T, 1024, MODE, Z3>(a, sI, tile, sm, red, rf); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// adjoint stage.  Staged by bulk copies: the packed spectrum of N * Bbar_s
// (barrier 0) and, with one halo row on each side, Y_s, Bbar_s and psi, plus
// the pointwise rows of lambda, gpart, G, the dJ/dpsi Kahan pair and Y, B of
// the next stage (barrier 1).  Shared memory: [scratch kExch complex]
// [Y_s halo][Bbar halo][psi halo][17 pointwise arrays x R rows]
// [W_{2L}^k, k < 2L].
// ---------------------------------------------------------------------------

// Conversions between a node value (T) and the frequency domain's real
// type (S): identity, or the double-float pair of an FP32 value and back.
template <typename T> __device__ __forceinline__ T spec_to(T v) { return v; }
template <typename T> __device__ __forceinline__ T spec_to(dfloat v) { return v.to_float(); }
template <typename T> __device__ __forceinline__ T spec_to(double v) { return (T)v; }
template <typename S, typename T> __device__ __forceinline__ S spec_from(T v) { return S(v); }

// SPLIT: the node phase alone -- the demag transpose comes from a.Dext and
// no row transform runs here (its own launches do them); shared memory then
// holds only the staged halo rows.
template <typename T, typename S, int L, bool Z3, bool DP, bool SPLIT = false>
__device__ __forceinline__ void adj_body(const AdjArgs<T, S>& a, const DevInst& I, const RowTile& tile,
                                         unsigned char* smem_raw, uint64_t* bars) {
  using C = cplx<S>;
  using G = RowGeom<L>;
  constexpr int RM = G::RM;
  constexpr int GS = seq_group_stride<C>(L);
  static_assert(rows_per_tile(L) * 3 * GS <= kExch, "row slots fit the exchange scratch");
  const G g(threadIdx.x);
  const int tid = threadIdx.x;
  const int nr = tile.nrows;
  const bool active = g.rl < nr;
  const int nx = I.nx, ny = I.ny, y0 = tile.y0;
  const int y = y0 + (active ? g.rl : 0);
  const int z = tile.z, nz = I.nz;
  const long long nodes = I.nodes, layer = I.layer;
  const long long zoff = (long long)z * layer;   // first node of the tile's layer
  C* sx = reinterpret_cast<C*>(smem_raw);
  T* sYs = SPLIT ? reinterpret_cast<T*>(smem_raw) : reinterpret_cast<T*>(sx + kExch);
  T* sBb = sYs + 3 * (RM + 2) * nx;
  T* sP = sBb + 3 * (RM + 2) * nx;
  C* tw2 = reinterpret_cast<C*>(sP + (RM + 2) * nx);
  C* sE = sx + g.rl * 3 * GS;
  C* grp = sE + g.c * GS;
  S* sEr = reinterpret_cast<S*>(sE);
  C* row0 = SPLIT ? nullptr : a.spec + I.spec_off + ((long long)z * ny + y0) * 3 * L;
  const long long n = (a.step_base ? *a.step_base : 0) + a.local_step;
  const int s = a.stage;
  const long long off3 = 3 * I.node_off;
  const Coef<T>& K = coef<T>(I);
  const T Ms = K.Ms, cx = K.cx, cy = K.cy, cz = K.cz, kan = K.kan;
  const T ku[3] = {K.ku[0], K.ku[1], K.ku[2]};
  const T dt = (T)a.dt;
  T ca = 0, cb = 0;   // u_{s-1} = ca lambda + cb g_s
  // Dormand-Prince: this instance's step size (0: idle in this reverse step)
  const T hdp = DP ? (T)a.hst[4 * tile.inst + 1] : (T)0;
  // per-step adjoint weights of the spectral and curve objectives at stage 1
  // of step n: one pair per block, converted once (no FP64 work per node)
  T ow0 = 0, ow1 = 0;
  if (!DP && s == 1 && a.wtab && ((I.objective == 2 && n >= a.n_from) || I.objective == 3)) {
    ow0 = (T)a.wtab[I.wt_off + 2 * n];
    ow1 = (T)a.wtab[I.wt_off + 2 * n + 1];
  }
  if (s == 4) { ca = dt / (T)3; cb = dt; }
  else if (s == 3) { ca = dt / (T)3; cb = (T)0.5 * dt; }
  else if (s == 2) { ca = dt / (T)6; cb = (T)0.5 * dt; }
  const bool emit = a.seed_only || s > 1 || a.seed_next;
  const bool seed = a.seed_only != 0;
  T* __restrict__ glam = a.lam;
  T* __restrict__ gG = a.G;
  T* __restrict__ ggp = a.gpart;
  T* __restrict__ gpsib = a.psib;
  T* __restrict__ gpsic = a.psic;
  T* __restrict__ gbo = a.BbarOut;
  const T* __restrict__ gYp = a.Yprev;
  const T* __restrict__ gBp = a.Bprev;
  const int ylo = max(0, y0 - 1), yhi = min(ny, y0 + nr + 1);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  if (!SPLIT) load_row_twiddles<C, L>(tw2, a.tw);
  __syncthreads();
  if (tid == 0) {
    unsigned bytes = 0;
    if (!seed) {
      if (!SPLIT) {
        const unsigned rowb = (unsigned)(L * sizeof(C));
        mbar_arrive_expect(&bars[0], nr * 3 * rowb);
        for (int r = 0; r < nr; ++r)
          for (int c = 0; c < 3; ++c) bulk_load(sx + (r * 3 + c) * GS, row0 + (r * 3 + c) * L, rowb, &bars[0]);
      }
      const unsigned hb = (unsigned)((yhi - ylo) * nx * sizeof(T));
      bytes += 7 * hb;
    }
    mbar_arrive_expect(&bars[1], bytes);
    if (!seed) {
      stage_halo(sYs, RM, a.Ys + off3 + zoff, nodes, 3, nx, y0, ylo, yhi, &bars[1]);
      stage_halo(sBb, RM, a.Bbar + off3 + zoff, nodes, 3, nx, y0, ylo, yhi, &bars[1]);
      stage_halo(sP, RM, a.psi + I.node_off + zoff, nodes, 1, nx, y0, ylo, yhi, &bars[1]);
    }
  }
  if (!seed && !SPLIT) {
    mbar_wait(&bars[0], 0, a.err);
    C v[8];
    row_inverse_comp<S, L>(v, grp, active, grp, g.t, tw2);
  }
  mbar_wait(&bars[1], 0, a.err);
  __syncthreads();

  const int cs = (RM + 2) * nx;
  const T cc[4] = {cx, cx, cy, cy};
#pragma unroll 1
  for (int x = g.tr; active && x < nx; x += 3 * G::TT) {
    const long long n0 = zoff + (long long)y * nx + x;
    const int sl = node_slot<S, L>(x);
    // every pointwise value of this node first, so that the load latencies
    // overlap (these arrays are disjoint from the ones this loop writes)
    T lam[3], gg[3], gsum[3], yp[3], bp[3], dx[3];
    T qs = 0, qc = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = off3 + c * nodes + n0;
      lam[c] = glam[id];
      if (!seed) {
        gg[c] = ggp[id];
        gsum[c] = (!DP && s < 4) ? gG[id] : (T)0;
        if (SPLIT) dx[c] = a.Dext[id];
      }
      if (emit) {
        yp[c] = gYp[id];
        bp[c] = gBp[id];
      }
    }
    if (!seed) {
      qs = gpsib[I.node_off + n0];
      qc = gpsic[I.node_off + n0];
    }
    T u[3];
    if (seed) {
#pragma unroll
      for (int c = 0; c < 3; ++c) u[c] = DP ? hdp * a.dpb * lam[c] : dt / (T)6 * lam[c];
    } else {
      const int oi = (g.rl + 1) * nx + x;
      const T pi = sP[oi];
      T yi[3], bi[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        yi[c] = sYs[c * cs + oi];
        bi[c] = sBb[c * cs + oi];
      }
      T qpsi = 0;
      // exchange transpose (gather form) and its psi derivative
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const bool ok = d == 0 ? x + 1 < nx : d == 1 ? x > 0 : d == 2 ? y + 1 < ny : y > 0;
        if (!ok) continue;
        const int oj = oi + (d == 0 ? 1 : d == 1 ? -1 : d == 2 ? nx : -nx);
        const T pj = sP[oj];
        const T sp = pi + pj;
        const T r = sp > (T)0 ? (T)1 / sp : (T)0;
        const T wij = (T)2 * pj * r, wji = (T)2 * pi * r;   // edge weights seen by i and by j
        T eij = 0, eji = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T yj = sYs[c * cs + oj], bj = sBb[c * cs + oj];
          gg[c] += cc[d] * (wji * bj - wij * bi[c]);
          eij += bi[c] * (yj - yi[c]);
          eji += bj * (yi[c] - yj);
        }
        qpsi += cc[d] * wij * r * (eji - eij);          // d w_ij/d psi_i = -2 psi_j/(psi_i+psi_j)^2
      }
      // the same across the layers above and below (3D), from global memory
      if constexpr (Z3) {
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        if (d == 0 ? z + 1 >= nz : z == 0) continue;
        const long long j = n0 + (d == 0 ? layer : -layer);
        const T pj = a.psi[I.node_off + j];
        const T sp = pi + pj;
        const T r = sp > (T)0 ? (T)1 / sp : (T)0;
        const T wij = (T)2 * pj * r, wji = (T)2 * pi * r;
        T eij = 0, eji = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T yj = a.Ys[off3 + c * nodes + j], bj = a.Bbar[off3 + c * nodes + j];
          gg[c] += cz * (wji * bj - wij * bi[c]);
          eij += bi[c] * (yj - yi[c]);
          eji += bj * (yi[c] - yj);
        }
        qpsi += cz * wij * r * (eji - eij);
      }
      }
      // demag transpose Ms psi_i (N * Bbar)_i and its psi derivative
      T D[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        D[c] = SPLIT ? dx[c] : spec_to<T>(sEr[2 * c * GS + sl]);
        gg[c] += Ms * pi * D[c];
      }
      qpsi += Ms * dot3(yi, D);
      if (s == 1 && I.objective == 3) {
        // curve sample at step n: the quotient-rule term of P = sum psi m / sum psi
        qpsi += ow0 * yi[I.comp] - ow1;
      }
      kahan_add(qs, qc, qpsi);
      gpsib[I.node_off + n0] = qs;
      gpsic[I.node_off + n0] = qc;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long id = off3 + c * nodes + n0;
        if constexpr (DP) {
          // eta_s to its slot; at stage 1 lambda_k = lambda_{k+1} + sum_s eta_s
          a.ebuf[(long long)(s - 1) * a.kstride + id] = gg[c];
          if (s == 1) {
            T sum = gg[c];
            for (int i = 2; i <= 6; ++i) sum += a.ebuf[(long long)(i - 1) * a.kstride + id];
            lam[c] += sum;
          }
        } else if (s == 4) {
          gG[id] = gg[c];
        } else if (s > 1) {
          gG[id] = gsum[c] + gg[c];
        } else {
          lam[c] += gsum[c] + gg[c];
        }
      }
      if (s == 1) {
        if (I.objective == 0 && n >= a.n_from) {
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            if (!in_box(I.boxes[b], x, y)) continue;
            const T vv = yi[I.comp];
            lam[I.comp] += K.wbox[b] * (I.power == 2 ? (T)2 * vv : (T)1);
          }
        } else if (I.objective == 2 && n >= a.n_from) {
          if (in_box(I.boxes[0], x, y)) lam[I.comp] += ow0;
          if (in_box(I.boxes[1], x, y)) lam[I.comp] += ow1;
        } else if (I.objective == 3) {
          lam[I.comp] += ow0 * pi;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) glam[off3 + c * nodes + n0] = lam[c];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if constexpr (DP) {
          // kappa_{s-1} = h (b_{s-1} lambda + sum_{i >= s} a(i, s-1) eta_i)
          T kap = a.dpb * lam[c] + a.dpa[s] * gg[c];
          const long long id = off3 + c * nodes + n0;
          for (int i = s + 1; i <= 6; ++i)
            if (a.dpa[i] != (T)0) kap += a.dpa[i] * a.ebuf[(long long)(i - 1) * a.kstride + id];
          u[c] = hdp * kap;
        } else {
          u[c] = (s > 1) ? ca * lam[c] + cb * gg[c] : dt / (T)6 * lam[c];
        }
      }
    }
    if (!emit) continue;
    T bbar[3], gl[3], al, ga;
    damping_at(I, K, x, y, al, ga);
    rhs_vjp(u, yp, bp, al, ga, bbar, gl);
    if (kan != (T)0) {
      const T dd = dot3(bbar, ku);
#pragma unroll
      for (int c = 0; c < 3; ++c) gl[c] += kan * dd * ku[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = off3 + c * nodes + n0;
      gbo[id] = bbar[c];
      ggp[id] = gl[c];
      if (!SPLIT) sEr[2 * c * GS + sl] = spec_from<S>(bbar[c]);
    }
  }
  if (!emit || SPLIT) return;
  __syncthreads();
  row_forward_comp<S, L>(grp, nx / 2, a.spec + I.spec_off + ((long long)z * ny + y) * 3 * L + g.c * L, active, g.t,
                         tw2);
}

template <typename T, typename S, bool Z3, bool DP, bool SPLIT = false>
__device__ __forceinline__ void adj_dispatch(const AdjArgs<T, S>& a, const DevInst& I, const RowTile& tile,
                                             unsigned char* smem_raw, uint64_t* bars) {
  switch (I.log2Lx) {
    case 3: adj_body<T, S, 8, Z3, DP, SPLIT>(a, I, tile, smem_raw, bars); break;
    case 4: adj_body<T, S, 16, Z3, DP, SPLIT>(a, I, tile, smem_raw, bars); break;
    case 5: adj_body<T, S, 32, Z3, DP, SPLIT>(a, I, tile, smem_raw, bars); break;
    case 6: adj_body<T, S, 64, Z3, DP, SPLIT>(a, I, tile, smem_raw, bars); break;
    case 7: adj_body<T, S, 128, Z3, DP, SPLIT>(a, I, tile, smem_raw, bars); break;
    case 8: adj_body<T, S, 256, Z3, DP, SPLIT>(a, I, tile, smem_raw, bars); break;
    case 9: adj_body<T, S, 512, Z3, DP, SPLIT>(a, I, tile, smem_raw, bars); break;
    case 10: adj_body<T, S, 1024, Z3, DP, SPLIT>(a, I, tile, smem_raw, bars); break;
    default: break;
  }
}

// MB: blocks per SM the adjoint stage kernel is compiled for: FP32 2;
// FP64 1; FP32 with a double-float frequency domain 1 or 2 (candidates).
template <typename T, typename S, bool Z3, int MB>
__global__ void __launch_bounds__(kAdjThreads, MB) adj_kernel(AdjArgs<T, S> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevInst sI;
  __shared__ uint64_t bars[2];
  const RowTile tile = a.tiles[blockIdx.x];
  load_inst(sI, a.inst + tile.inst);
  __syncthreads();
  adj_dispatch<T, S, Z3, false>(a, sI, tile, smem_raw, bars);
}

// node phase of a film adjoint stage whose row transforms run as their own
// launches (shared memory holds only the halo rows); MB: 2 or 3 blocks per
// SM (80 or 56 registers, the latter with spills: a launch candidate)
template <typename T, int MB>
__global__ void __launch_bounds__(kAdjThreads, MB) adj_split_kernel(AdjArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevInst sI;
  __shared__ uint64_t bars[2];
  const RowTile tile = a.tiles[blockIdx.x];
  load_inst(sI, a.inst + tile.inst);
  __syncthreads();
  adj_dispatch<T, T, false, false, true>(a, sI, tile, smem_raw, bars);
}

// ---------------------------------------------------------------------------
// row transforms of a frequency domain as launches of their own (used with
// the split adjoint stage): one row tile per block, the same thread layout
// as the row-family kernels.  DIR = +1: bulk copy of the tile's spectrum
// rows, inverse row FFT, the field at the nodes to `out`; DIR = -1: the
// nodes' values from `src`, forward row FFT, packed rows to the spectrum.
// Shared memory: exchange scratch (kExch complex of S) and W_{2L}.
// ---------------------------------------------------------------------------

template <typename T, typename S, int L, int DIR>
__device__ __forceinline__ void spec_rows_body(const SpecRowArgs<T, S>& a, const DevInst& I, const RowTile& tile,
                                               unsigned char* smem_raw, uint64_t* bar) {
  using C = cplx<S>;
  using G = RowGeom<L>;
  constexpr int GS = seq_group_stride<C>(L);
  static_assert(rows_per_tile(L) * 3 * GS <= kExch, "row slots fit the exchange scratch");
  const G g(threadIdx.x);
  const int nr = tile.nrows;
  const bool active = g.rl < nr;
  const int nx = I.nx, ny = I.ny, y0 = tile.y0;
  const int y = y0 + (active ? g.rl : 0);
  const long long nodes = I.nodes;
  const long long zoff = (long long)tile.z * I.layer;
  C* sx = reinterpret_cast<C*>(smem_raw);
  C* tw2 = sx + kExch;
  C* sE = sx + g.rl * 3 * GS;
  C* grp = sE + g.c * GS;
  S* sEr = reinterpret_cast<S*>(sE);
  C* row0 = a.spec + I.spec_off + ((long long)tile.z * ny + y0) * 3 * L;
  const long long off3 = 3 * I.node_off;
  if (DIR > 0 && threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  load_row_twiddles<C, L>(tw2, a.tw);
  __syncthreads();
  if (DIR > 0) {
    if (threadIdx.x == 0) {
      const unsigned rowb = (unsigned)(L * sizeof(C));
      mbar_arrive_expect(bar, nr * 3 * rowb);
      for (int r = 0; r < nr; ++r)
        for (int c = 0; c < 3; ++c) bulk_load(sx + (r * 3 + c) * GS, row0 + (r * 3 + c) * L, rowb, bar);
    }
    mbar_wait(bar, 0, a.err);
    C v[8];
    row_inverse_comp<S, L>(v, grp, active, grp, g.t, tw2);
    __syncthreads();
#pragma unroll 1
    for (int x = g.tr; active && x < nx; x += 3 * G::TT) {
      const long long n0 = zoff + (long long)y * nx + x;
      const int sl = node_slot<S, L>(x);
#pragma unroll
      for (int c = 0; c < 3; ++c) a.out[off3 + c * nodes + n0] = spec_to<T>(sEr[2 * c * GS + sl]);
    }
  } else {
#pragma unroll 1
    for (int x = g.tr; active && x < nx; x += 3 * G::TT) {
      const long long n0 = zoff + (long long)y * nx + x;
      const int sl = node_slot<S, L>(x);
#pragma unroll
      for (int c = 0; c < 3; ++c) sEr[2 * c * GS + sl] = spec_from<S>(a.src[off3 + c * nodes + n0]);
    }
    __syncthreads();
    row_forward_comp<S, L>(grp, nx / 2, a.spec + I.spec_off + ((long long)tile.z * ny + y) * 3 * L + g.c * L,
                           active, g.t, tw2);
  }
}

template <typename T, typename S, int DIR>
__global__ void __launch_bounds__(kRowThreads, 2) spec_rows_kernel(SpecRowArgs<T, S> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevInst sI;
  __shared__ uint64_t bar;
  const RowTile tile = a.tiles[blockIdx.x];
  load_inst(sI, a.inst + tile.inst);
  __syncthreads();
  switch (sI.log2Lx) {
    case 3: spec_rows_body<T, S, 8, DIR>(a, sI, tile, smem_raw, &bar); break;
    case 4: spec_rows_body<T, S, 16, DIR>(a, sI, tile, smem_raw, &bar); break;
    case 5: spec_rows_body<T, S, 32, DIR>(a, sI, tile, smem_raw, &bar); break;
    case 6: spec_rows_body<T, S, 64, DIR>(a, sI, tile, smem_raw, &bar); break;
    case 7: spec_rows_body<T, S, 128, DIR>(a, sI, tile, smem_raw, &bar); break;
    case 8: spec_rows_body<T, S, 256, DIR>(a, sI, tile, smem_raw, &bar); break;
    case 9: spec_rows_body<T, S, 512, DIR>(a, sI, tile, smem_raw, &bar); break;
    case 10: spec_rows_body<T, S, 1024, DIR>(a, sI, tile, smem_raw, &bar); break;
    default: break;
  }
}

// adjoint stage of a Dormand-Prince step (stages 6..1; the seed at stage 6)
template <typename T, bool Z3>
__global__ void __launch_bounds__(kAdjThreads, sizeof(T) == 4 ? 2 : 1) adj_dp_kernel(AdjArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevInst sI;
  __shared__ uint64_t bars[2];
  const RowTile tile = a.tiles[blockIdx.x];
  load_inst(sI, a.inst + tile.inst);
  __syncthreads();
  adj_dispatch<T, T, Z3, true>(a, sI, tile, smem_raw, bars);
}

// ---------------------------------------------------------------------------
// elementwise kernels (one CTA per row tile)
// ---------------------------------------------------------------------------

template <typename T>
__global__ void material_kernel(const DevInst* inst, const RowTile* tiles, const T* phi, T* psi, T* dpsi,
                                double* psitile, double* psimom) {
  __shared__ double red[32];
  const RowTile tile = tiles[blockIdx.x];
  const DevInst& I = inst[tile.inst];
  const long long base = tile_base(I, tile);
  const int cnt = tile.nrows * I.nx;
  double acc = 0.0, ax = 0.0, ay = 0.0;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const double ph = (double)phi[base + e];
    const double p = 1.0 / (1.0 + exp(-I.sigmoid_a * ph));   // Eq. 4
    psi[base + e] = (T)p;
    dpsi[base + e] = (T)(I.sigmoid_a * p * (1.0 - p));
    acc += p;
    ax += p * (double)(e % I.nx);                             // psi-weighted node index (x, y)
    ay += p * (double)(tile.y0 + e / I.nx);
  }
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) psitile[I.tile_off + tile.k] = tot;
  if (psimom) {
    __syncthreads();
    const double sx = block_sum(ax, red);
    if (threadIdx.x == 0) psimom[2 * (I.tile_off + tile.k)] = sx;
    __syncthreads();
    const double sy = block_sum(ay, red);
    if (threadIdx.x == 0) psimom[2 * (I.tile_off + tile.k) + 1] = sy;
  }
}

// dJ/dPhi = a psi (1 - psi) (sum - compensation) of the Kahan pair, times the
// instance's cotangent w (nullable: 1); with dm0 also dJ/dm0 = w lambda_0.
template <typename T>
__global__ void grad_finish_kernel(const DevInst* inst, const RowTile* tiles, const T* dpsi, const T* psib,
                                   const T* psic, const double* w, T* out, const T* lam, T* dm0) {
  const RowTile tile = tiles[blockIdx.x];
  const DevInst& I = inst[tile.inst];
  const long long base = tile_base(I, tile);
  const int cnt = tile.nrows * I.nx;
  const double wi = w ? w[tile.inst] : 1.0;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const double g = ((double)psib[base + e] - (double)psic[base + e]) * (double)dpsi[base + e];
    out[base + e] = (T)(wi * g);
  }
  if (!dm0) return;
  for (int c = 0; c < 3; ++c)
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const long long id = 3 * I.node_off + (long long)c * I.nodes + (base - I.node_off) + e;
      dm0[id] = w ? (T)(wi * (double)lam[id]) : lam[id];
    }
}

__device__ __forceinline__ void atomic_max_abs(unsigned int* p, float v) {
  atomicMax(p, __float_as_uint(fabsf(v)));
}
__device__ __forceinline__ void atomic_max_abs(unsigned int* p, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(fabs(v)));
}

template <typename T>
__global__ void levelset_update_kernel(const DevInst* inst, const RowTile* tiles, T* phi, const T* grad,
                                       const unsigned char* mask, T lr, unsigned int* maxbits) {
  const RowTile tile = tiles[blockIdx.x];
  const DevInst& I = inst[tile.inst];
  const long long base = tile_base(I, tile);
  const int cnt = tile.nrows * I.nx;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    if (!mask[base + e]) continue;
    const T v = phi[base + e] - lr * grad[base + e];   // Eq. 5
    phi[base + e] = v;
    atomic_max_abs(maxbits + 2 * tile.inst, v);
  }
}

__device__ __forceinline__ float max_from_bits(const unsigned int* p, float*) { return __uint_as_float(*p); }
__device__ __forceinline__ double max_from_bits(const unsigned int* p, double*) {
  return __longlong_as_double((long long)*reinterpret_cast<const unsigned long long*>(p));
}

template <typename T>
__global__ void levelset_scale_kernel(const DevInst* inst, const RowTile* tiles, T* phi,
                                      const unsigned char* mask, const unsigned int* maxbits) {
  const RowTile tile = tiles[blockIdx.x];
  const DevInst& I = inst[tile.inst];
  const long long base = tile_base(I, tile);
  const int cnt = tile.nrows * I.nx;
  const T mx = max_from_bits(maxbits + 2 * tile.inst, (T*)nullptr);
  if (!(mx > (T)0)) return;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x)
    if (mask[base + e]) phi[base + e] = phi[base + e] / mx;   // renormalise to [-1, 1]
}

// ---------------------------------------------------------------------------
// launch helpers, instantiated per precision and kernel family in the k_*.cu
// translation units (compiled in parallel)
// ---------------------------------------------------------------------------

template <typename T, int MODE>
void launch_rows_mode(const RowArgs<T>& a, int ntiles, size_t smem, cudaStream_t st, bool z3) {
  if (z3) rows_kernel<T, MODE, true><<<ntiles, kRowThreads, smem, st>>>(a);
  else rows_kernel<T, MODE, false><<<ntiles, kRowThreads, smem, st>>>(a);
}
// The dynamic shared-memory limit is a process-wide attribute of each kernel:
// it is only ever raised, so that a context for small grids does not lower it
// below what another context (or llg_field_noalloc) launches with.
inline void raise_smem_limit(const void* fn, size_t* cur, size_t smem) {
  if (smem > *cur) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    *cur = smem;
  }
}
template <typename T, int MODE>
void smem_rows_mode(size_t smem) {
  static size_t cur = 0, cur3 = 0;
  raise_smem_limit(reinterpret_cast<const void*>(rows_kernel<T, MODE, false>), &cur, smem);
  raise_smem_limit(reinterpret_cast<const void*>(rows_kernel<T, MODE, true>), &cur3, smem);
}
// Register-cap variants compiled per type: the first is the default.
template <typename T> struct Variants { static constexpr int a = 1, b = 1; };
template <> struct Variants<float> { static constexpr int a = 3, b = 3; };
template <> struct Variants<dfloat> { static constexpr int a = 2, b = 1; };
template <typename T, typename S> struct AdjVariants { static constexpr int a = 1, b = 1; };
template <> struct AdjVariants<float, float> { static constexpr int a = 2, b = 2; };
template <> struct AdjVariants<float, dfloat> { static constexpr int a = 2, b = 1; };

template <typename T>
void launch_cols(const ColArgs<T>& a, int ntiles, size_t smem, cudaStream_t st, int mb) {
  if (mb == Variants<T>::b) cols_kernel<T, Variants<T>::b><<<ntiles, kColThreads, smem, st>>>(a);
  else cols_kernel<T, Variants<T>::a><<<ntiles, kColThreads, smem, st>>>(a);
}
template <typename T>
void smem_cols(size_t smem) {
  static size_t cur = 0, cur2 = 0;
  raise_smem_limit(reinterpret_cast<const void*>(cols_kernel<T, Variants<T>::a>), &cur, smem);
  raise_smem_limit(reinterpret_cast<const void*>(cols_kernel<T, Variants<T>::b>), &cur2, smem);
}
template <typename T, typename S>
void launch_adj(const AdjArgs<T, S>& a, int ntiles, size_t smem, cudaStream_t st, bool z3, int mb) {
  constexpr int A = AdjVariants<T, S>::a, B = AdjVariants<T, S>::b;
  if (mb == B && B != A) {
    if (z3) adj_kernel<T, S, true, B><<<ntiles, kAdjThreads, smem, st>>>(a);
    else adj_kernel<T, S, false, B><<<ntiles, kAdjThreads, smem, st>>>(a);
  } else {
    if (z3) adj_kernel<T, S, true, A><<<ntiles, kAdjThreads, smem, st>>>(a);
    else adj_kernel<T, S, false, A><<<ntiles, kAdjThreads, smem, st>>>(a);
  }
}
template <typename T, typename S>
void smem_adj(size_t smem) {
  constexpr int A = AdjVariants<T, S>::a, B = AdjVariants<T, S>::b;
  static size_t cur[4] = {0, 0, 0, 0};
  raise_smem_limit(reinterpret_cast<const void*>(adj_kernel<T, S, false, A>), &cur[0], smem);
  raise_smem_limit(reinterpret_cast<const void*>(adj_kernel<T, S, true, A>), &cur[1], smem);
  raise_smem_limit(reinterpret_cast<const void*>(adj_kernel<T, S, false, B>), &cur[2], smem);
  raise_smem_limit(reinterpret_cast<const void*>(adj_kernel<T, S, true, B>), &cur[3], smem);
}
template <typename T>
void launch_adj_split(const AdjArgs<T>& a, int ntiles, size_t smem, cudaStream_t st, int mb) {
  if (mb == 3) adj_split_kernel<T, 3><<<ntiles, kAdjThreads, smem, st>>>(a);
  else adj_split_kernel<T, 2><<<ntiles, kAdjThreads, smem, st>>>(a);
}
template <typename T>
void smem_adj_split(size_t smem) {
  static size_t cur = 0, cur3 = 0;
  raise_smem_limit(reinterpret_cast<const void*>(adj_split_kernel<T, 2>), &cur, smem);
  raise_smem_limit(reinterpret_cast<const void*>(adj_split_kernel<T, 3>), &cur3, smem);
}
template <typename T, typename S>
void launch_spec_rows(const SpecRowArgs<T, S>& a, int dir, int ntiles, size_t smem, cudaStream_t st) {
  if (dir > 0) spec_rows_kernel<T, S, 1><<<ntiles, kRowThreads, smem, st>>>(a);
  else spec_rows_kernel<T, S, -1><<<ntiles, kRowThreads, smem, st>>>(a);
}
template <typename T, typename S>
void smem_spec_rows(size_t smem) {
  static size_t cur = 0, cur2 = 0;
  raise_smem_limit(reinterpret_cast<const void*>(spec_rows_kernel<T, S, 1>), &cur, smem);
  raise_smem_limit(reinterpret_cast<const void*>(spec_rows_kernel<T, S, -1>), &cur2, smem);
}
template <typename T>
void launch_adj_dp(const AdjArgs<T>& a, int ntiles, size_t smem, cudaStream_t st, bool z3) {
  if (z3) adj_dp_kernel<T, true><<<ntiles, kAdjThreads, smem, st>>>(a);
  else adj_dp_kernel<T, false><<<ntiles, kAdjThreads, smem, st>>>(a);
}
template <typename T>
void smem_adj_dp(size_t smem) {
  static size_t cur = 0, cur3 = 0;
  raise_smem_limit(reinterpret_cast<const void*>(adj_dp_kernel<T, false>), &cur, smem);
  raise_smem_limit(reinterpret_cast<const void*>(adj_dp_kernel<T, true>), &cur3, smem);
}

// Dormand-Prince reverse sweep: the state m_k of each instance's step being
// reversed, from its checkpoint slot (slot[inst] < 0: idle, nothing copied)
template <typename T>
__global__ void dp_gather_kernel(const DevInst* inst, const RowTile* tiles, const T* ckall, long long kstride,
                                 const long long* slot, T* out) {
  const RowTile tile = tiles[blockIdx.x];
  const DevInst& I = inst[tile.inst];
  const long long k = slot[tile.inst];
  if (k < 0) return;
  const long long base = tile_base(I, tile);
  const int cnt = tile.nrows * I.nx;
  for (int c = 0; c < 3; ++c)
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const long long id = 3 * I.node_off + (long long)c * I.nodes + (base - I.node_off) + e;
      out[id] = ckall[k * kstride + id];
    }
}
template <typename T>
void launch_dp_gather(const DevInst* inst, const RowTile* tiles, int ntiles, const T* ckall, long long kstride,
                      const long long* slot, T* out, cudaStream_t st) {
  dp_gather_kernel<T><<<ntiles, 256, 0, st>>>(inst, tiles, ckall, kstride, slot, out);
}

// Dormand-Prince replay: src (the state after replay step *jptr) to segment
// slot j + 1 and to the working state mrev (src may be mrev itself)
template <typename T>
__global__ void dp_push_kernel(const DevInst* inst, const RowTile* tiles, const T* src, T* seg, long long kstride,
                               const long long* jptr, T* mrev) {
  const RowTile tile = tiles[blockIdx.x];
  const DevInst& I = inst[tile.inst];
  const long long j1 = *jptr + 1;
  const long long base = tile_base(I, tile);
  const int cnt = tile.nrows * I.nx;
  for (int c = 0; c < 3; ++c)
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const long long id = 3 * I.node_off + (long long)c * I.nodes + (base - I.node_off) + e;
      const T v = src[id];
      seg[j1 * kstride + id] = v;
      mrev[id] = v;
    }
}
template <typename T>
void launch_dp_push(const DevInst* inst, const RowTile* tiles, int ntiles, const T* src, T* seg, long long kstride,
                    const long long* jptr, T* mrev, cudaStream_t st) {
  dp_push_kernel<T><<<ntiles, 256, 0, st>>>(inst, tiles, src, seg, kstride, jptr, mrev);
}
template <typename T>
void launch_material_tiles(const DevInst* inst, const RowTile* tiles, int ntiles, const T* phi, T* psi,
                           T* dpsi, double* psitile, double* psimom, cudaStream_t st) {
  material_kernel<T><<<ntiles, 256, 0, st>>>(inst, tiles, phi, psi, dpsi, psitile, psimom);
}
template <typename T>
void launch_grad_finish_tiles(const DevInst* inst, const RowTile* tiles, int ntiles, const T* dpsi,
                              const T* psib, const T* psic, const double* w, T* out, const T* lam, T* dm0,
                              cudaStream_t st) {
  grad_finish_kernel<T><<<ntiles, 256, 0, st>>>(inst, tiles, dpsi, psib, psic, w, out, lam, dm0);
}
template <typename T>
void launch_levelset_tiles(const DevInst* inst, const RowTile* tiles, int ntiles, T* phi, const T* grad,
                           const unsigned char* mask, double lr, unsigned int* maxbits, cudaStream_t st) {
  levelset_update_kernel<T><<<ntiles, 256, 0, st>>>(inst, tiles, phi, grad, mask, (T)lr, maxbits);
  levelset_scale_kernel<T><<<ntiles, 256, 0, st>>>(inst, tiles, phi, mask, maxbits);
}

}  // namespace llg
