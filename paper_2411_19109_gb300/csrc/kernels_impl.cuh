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
#include "tma.cuh"

namespace llg {

constexpr int kRowThreads = 128;
constexpr int kColThreads = 128;
constexpr int kAdjThreads = 128;



// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T edge_weight(T pi, T pj) {
  // w_ij = 2 psi_j/(psi_i + psi_j): harmonic-mean exchange coupling seen by i
  const T s = pi + pj;
  return s > (T)0 ? (T)2 * pj / s : (T)0;
}

template <typename T>
__device__ __forceinline__ T alpha_at(const DevInst& I, int x, int y) {
  const T a0 = (T)I.alpha;
  if (I.absorb_nodes <= 0) return a0;
  int d = INT_MAX;
  if (I.absorb_x) d = min(d, min(x, I.nx - 1 - x));
  if (I.absorb_y) d = min(d, min(y, I.ny - 1 - y));
  if (d == INT_MAX) return a0;
  const T W = (T)I.absorb_nodes;
  const T ramp = fmax((T)0, (W - (T)d) / W);
  return a0 + ((T)I.alpha_edge - a0) * ramp;
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

// LL form of Eq. 11: k = -gamma/(1+a^2) [Y x B + a Y x (Y x B)]
template <typename T>
__device__ __forceinline__ void llg_rhs(const T Y[3], const T B[3], T a, T k[3]) {
  const T g = -(T)kGamma / ((T)1 + a * a);
  T c1[3], c2[3];
  cross3(Y, B, c1);
  cross3(Y, c1, c2);
  for (int c = 0; c < 3; ++c) k[c] = g * (c1[c] + a * c2[c]);
}

// Cotangents of k = f(Y, B) for a slope cotangent u:
//   Bbar = -g [u x Y + a((u.Y) Y - (Y.Y) u)]
//   mloc = -g [B x u + a((Y.B) u + (u.Y) B - 2 (u.B) Y)]
template <typename T>
__device__ __forceinline__ void rhs_vjp(const T u[3], const T Y[3], const T B[3], T a, T Bbar[3],
                                        T mloc[3]) {
  const T g = -(T)kGamma / ((T)1 + a * a);
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

// ---------------------------------------------------------------------------
// node-pair access helpers.  A thread owns the adjacent nodes x0 = 2j and
// x0 + 1 of one row, matching the complex slot z_j = (x[2j], x[2j+1]) of the
// packed real row FFT.  Pairs are 8-byte (FP32) / 16-byte (FP64) aligned.
// ---------------------------------------------------------------------------

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T>
__device__ __forceinline__ void ld2(const T* p, T& a, T& b) {
  const typename Vec2<T>::type v = *reinterpret_cast<const typename Vec2<T>::type*>(p);
  a = v.x;
  b = v.y;
}
template <typename T>
__device__ __forceinline__ void st2(T* p, T a, T b) {
  typename Vec2<T>::type v;
  v.x = a;
  v.y = b;
  *reinterpret_cast<typename Vec2<T>::type*>(p) = v;
}

// Neighbour data of a node pair: index 0 = node x0, 1 = node x0+1.
// nbr order: +x, -x, +y, -y.
template <typename T>
struct PairNbr {
  T y[2][3];          // own values
  T p[2];             // own psi
  T yn[2][4][3];      // neighbour values
  T pn[2][4];         // neighbour psi
  bool ok[2][4];      // neighbour exists
};

// Gather a 3-vector field F (layout [c][node]) and psi around the pair.
template <typename T>
__device__ __forceinline__ void gather_pair(const T* __restrict__ F, const T* __restrict__ ps, long long nodes,
                                            int nx, int ny, int x0, int y, PairNbr<T>& q) {
  const long long n0 = (long long)y * nx + x0;
  const bool has_l = x0 > 0, has_r = x0 + 2 < nx, has_u = y + 1 < ny, has_d = y > 0;
  ld2(ps + n0, q.p[0], q.p[1]);
  T pu0 = 0, pu1 = 0, pd0 = 0, pd1 = 0;
  if (has_u) ld2(ps + n0 + nx, pu0, pu1);
  if (has_d) ld2(ps + n0 - nx, pd0, pd1);
  const T pl = has_l ? ps[n0 - 1] : (T)0;
  const T pr = has_r ? ps[n0 + 2] : (T)0;
  q.pn[0][0] = q.p[1]; q.pn[0][1] = pl; q.pn[0][2] = pu0; q.pn[0][3] = pd0;
  q.pn[1][0] = pr;     q.pn[1][1] = q.p[0]; q.pn[1][2] = pu1; q.pn[1][3] = pd1;
  q.ok[0][0] = true;  q.ok[0][1] = has_l; q.ok[0][2] = has_u; q.ok[0][3] = has_d;
  q.ok[1][0] = has_r; q.ok[1][1] = true;  q.ok[1][2] = has_u; q.ok[1][3] = has_d;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T* Fc = F + c * nodes;
    ld2(Fc + n0, q.y[0][c], q.y[1][c]);
    T u0 = 0, u1 = 0, d0 = 0, d1 = 0;
    if (has_u) ld2(Fc + n0 + nx, u0, u1);
    if (has_d) ld2(Fc + n0 - nx, d0, d1);
    const T l = has_l ? Fc[n0 - 1] : (T)0;
    const T r = has_r ? Fc[n0 + 2] : (T)0;
    q.yn[0][0][c] = q.y[1][c]; q.yn[0][1][c] = l; q.yn[0][2][c] = u0; q.yn[0][3][c] = d0;
    q.yn[1][0][c] = r;         q.yn[1][1][c] = q.y[0][c]; q.yn[1][2][c] = u1; q.yn[1][3][c] = d1;
  }
}

// B_ex,i = sum_j c_d w_ij (Y_j - Y_i)
template <typename T>
__device__ __forceinline__ void exchange_node(const PairNbr<T>& q, int i, T cx, T cy, T B[3]) {
  const T cc[4] = {cx, cx, cy, cy};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    if (!q.ok[i][d]) continue;
    const T w = cc[d] * edge_weight(q.p[i], q.pn[i][d]);
#pragma unroll
    for (int c = 0; c < 3; ++c) B[c] += w * (q.yn[i][d][c] - q.y[i][c]);
  }
}

template <typename C>
__device__ __forceinline__ C unpack_one(const C* __restrict__ X, int kk, int L, const C* __restrict__ tw) {
  // Z[k] = (X_k + conj X_{L-k}) + i W_P^{-k} (X_k - conj X_{L-k}),  P = 2L
  const C xk = X[kk];
  if (kk == 0) return mk<C>(xk.x + xk.y, xk.x - xk.y);
  const C xm = cconj(X[L - kk]);
  C w = tw[kk * (kTwiddleN / (2 * L))];
  w.y = -w.y;
  return cadd(cadd(xk, xm), mul_pi(cmul(w, csub(xk, xm))));
}

template <typename C>
__device__ __forceinline__ C pack_one(C zk, C zm_conj, int kk, int L, const C* __restrict__ tw) {
  // X[k] = (Z_k + conj Z_{L-k})/2 - i W_P^k (Z_k - conj Z_{L-k})/2
  using R = decltype(C::x);
  if (kk == 0) return mk<C>(zk.x + zk.y, zk.x - zk.y);
  const C w = tw[kk * (kTwiddleN / (2 * L))];
  return cscale(cadd(cadd(zk, zm_conj), mul_mi(cmul(w, csub(zk, zm_conj)))), (R)0.5);
}

// Inverse row FFT of the three packed field spectra of one row into
// v[c][s] = (F_c[2j], F_c[2j+1]), j = t + TT s.
template <typename T, int L>
__device__ __forceinline__ void row_inverse(cplx<T> (&v)[3][8], const cplx<T>* __restrict__ row, bool active,
                                            cplx<T>* sm, int t, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int TT = L / 8;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int s = 0; s < 8; ++s)
      v[c][s] = active ? unpack_one(row + c * L, t + TT * s, L, tw) : mk<C>((T)0, (T)0);
  regfft<C, L, 1, 3>(v, sm, rf_padded_len(L), 1, t, tw);
}

// Forward row FFT of v[c][s] = (M_c[2j], M_c[2j+1]) and packed store.
template <typename T, int L>
__device__ __forceinline__ void row_forward(cplx<T> (&v)[3][8], cplx<T>* __restrict__ row, bool active,
                                            cplx<T>* sm, int t, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int TT = L / 8;
  constexpr int SP = rf_padded_len(L);
  regfft<C, L, -1, 3>(v, sm, SP, 1, t, tw);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int s = 0; s < 8; ++s) sm[c * SP + rf_pad(t + TT * s)] = v[c][s];
  __syncthreads();
  if (!active) return;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int kk = t + TT * s;
      const C zm = cconj(sm[c * SP + rf_pad((L - kk) & (L - 1))]);
      row[c * L + kk] = pack_one(v[c][s], zm, kk, L, tw);
    }
}

// ---------------------------------------------------------------------------
// column pass: FFT_y, product with the tensor spectrum, inverse FFT_y
// ---------------------------------------------------------------------------

__device__ __forceinline__ void load_tensor(const float* tab, long long idx, float n[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(tab) + idx);
  n[0] = v.x; n[1] = v.y; n[2] = v.z; n[3] = v.w;
}
__device__ __forceinline__ void load_tensor(const double* tab, long long idx, double n[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(tab) + 2 * idx);
  const double2 b = __ldg(reinterpret_cast<const double2*>(tab) + 2 * idx + 1);
  n[0] = a.x; n[1] = a.y; n[2] = b.x; n[3] = b.y;
}

template <typename T, int L>
__device__ __forceinline__ void cols_body(const ColArgs<T>& a, const DevInst& I, const ColTile& tile,
                                          cplx<T>* smem) {
  using C = cplx<T>;
  constexpr int TT = L / 8;
  constexpr int NC = (kColThreads / TT) > 0 ? kColThreads / TT : 1;   // columns per block
  constexpr int SP = rf_padded_len(L);
  const int tid = threadIdx.x;
  const int t = tid / NC, col = tid - t * NC;
  const bool active = col < tile.ncols;
  const int kx = tile.kx0 + (active ? col : 0);
  const int Lx = I.Lx, ny = I.ny;
  C* sm = smem + col;                    // element (c, i) of this column at sm[(c*SP + pad(i))*NC]
  C* spec = a.spec + I.spec_off;
  C v[3][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int y = t + TT * s;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      v[c][s] = (active && y < ny) ? spec[((long long)y * 3 + c) * Lx + kx] : mk<C>((T)0, (T)0);
  }
  regfft<C, L, -1, 3>(v, sm, SP, NC, t, a.tw);
  const bool dc_tile = tile.kx0 == 0;               // uniform over the block
  if (dc_tile) {
    if (col == 0)
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int s = 0; s < 8; ++s) sm[(c * SP + rf_pad(t + TT * s)) * NC] = v[c][s];
    __syncthreads();
  }
  const T* tab = a.tens + I.tens_off;
  constexpr int nky = L / 2 + 1;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int ky = t + TT * s;
    const bool lo = ky <= L / 2;
    const int kyf = lo ? ky : L - ky;
    if (kx != 0) {
      T n[4];
      load_tensor(tab, (long long)kx * nky + kyf, n);
      const T nxy = lo ? n[3] : -n[3];
      const C mx = v[0][s], my = v[1][s], mz = v[2][s];
      v[0][s] = mk<C>(n[0] * mx.x + nxy * my.x, n[0] * mx.y + nxy * my.y);
      v[1][s] = mk<C>(nxy * mx.x + n[1] * my.x, nxy * mx.y + n[1] * my.y);
      v[2][s] = mk<C>(n[2] * mz.x, n[2] * mz.y);
    } else {
      // packed DC (kx = 0) and Nyquist (kx = Px/2) columns: separate them by
      // Hermitian symmetry in ky, apply each its own (diagonal) tensor
      T nd[4], nq[4];
      load_tensor(tab, (long long)kyf, nd);
      load_tensor(tab, (long long)Lx * nky + kyf, nq);
      const int km = (L - ky) & (L - 1);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T p = (T)0.5 * (nd[c] + nq[c]), q = (T)0.5 * (nd[c] - nq[c]);
        const C vb = cconj(sm[(c * SP + rf_pad(km)) * NC]);
        v[c][s] = cadd(cscale(v[c][s], p), cscale(vb, q));
      }
    }
  }
  if (dc_tile) __syncthreads();
  regfft<C, L, 1, 3>(v, sm, SP, NC, t, a.tw);
  if (!active) return;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int y = t + TT * s;
    if (y < ny)
#pragma unroll
      for (int c = 0; c < 3; ++c) spec[((long long)y * 3 + c) * Lx + kx] = v[c][s];
  }
}

template <typename T>
__global__ void __launch_bounds__(kColThreads) cols_kernel(ColArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevInst sI;
  const ColTile tile = a.tiles[blockIdx.x];
  load_inst(sI, a.inst + tile.inst);
  __syncthreads();
  C* sm = reinterpret_cast<C*>(smem_raw);
  switch (sI.log2Py) {
    case 3: cols_body<T, 8>(a, sI, tile, sm); break;
    case 4: cols_body<T, 16>(a, sI, tile, sm); break;
    case 5: cols_body<T, 32>(a, sI, tile, sm); break;
    case 6: cols_body<T, 64>(a, sI, tile, sm); break;
    case 7: cols_body<T, 128>(a, sI, tile, sm); break;
    case 8: cols_body<T, 256>(a, sI, tile, sm); break;
    case 9: cols_body<T, 512>(a, sI, tile, sm); break;
    case 10: cols_body<T, 1024>(a, sI, tile, sm); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// row pass of the forward stage (and its variants)
// ---------------------------------------------------------------------------

template <typename T, int L, int MODE>
__device__ __forceinline__ void rows_body(const RowArgs<T>& a, const DevInst& I, const RowTile& tile,
                                          cplx<T>* smem, double* red, T rf) {
  using C = cplx<T>;
  constexpr int TT = L / 8;
  constexpr int SP = rf_padded_len(L);
  const int tid = threadIdx.x;
  const int rl = tid / TT, t = tid - rl * TT;
  const bool active = rl < tile.nrows;
  const int nx = I.nx, ny = I.ny;
  const int y = tile.y0 + (active ? rl : 0);
  const long long nodes = I.nodes;
  C* sm = smem + rl * 3 * SP;
  C* row = a.spec + I.spec_off + (long long)y * 3 * L;
  const long long n = (a.step_base ? *a.step_base : 0) + a.local_step;
  const int s = a.stage;
  const long long off3 = 3 * I.node_off;
  const T* __restrict__ Y = a.Yin + off3;
  const T* __restrict__ ps = a.psi + I.node_off;
  const T Ms = (T)I.Ms, cx = (T)I.cex_x, cy = (T)I.cex_y, kan = (T)I.kan;
  const T ku[3] = {(T)I.ku[0], (T)I.ku[1], (T)I.ku[2]};
  const T dt = (T)a.dt;

  C v[3][8];
  if (MODE != ROW_FFT_ONLY) row_inverse<T, L>(v, row, active, sm, t, a.tw);

  double vsum = 0.0;
  const bool objective_step = (MODE == ROW_STAGE) && s == 4 && a.slots != nullptr && I.objective == 0 &&
                              (n + 1) >= a.n_from;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int x0 = 2 * (t + TT * q);
    if (!active || x0 >= nx) {
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][q] = mk<C>((T)0, (T)0);
      continue;
    }
    const long long n0 = (long long)y * nx + x0;
    if (MODE == ROW_FFT_ONLY) {
      T p0, p1;
      ld2(ps + n0, p0, p1);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T a0, a1;
        ld2(Y + c * nodes + n0, a0, a1);
        v[c][q] = mk<C>(Ms * p0 * a0, Ms * p1 * a1);
      }
      continue;
    }
    T Bd[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Bd[0][c] = v[c][q].x;
      Bd[1][c] = v[c][q].y;
    }
    if (MODE == ROW_FIELD && a.demag_only) {
#pragma unroll
      for (int c = 0; c < 3; ++c) st2(a.Bout + off3 + c * nodes + n0, Bd[0][c], Bd[1][c]);
      continue;
    }
    PairNbr<T> P;
    gather_pair(Y, ps, nodes, nx, ny, x0, y, P);
    if (MODE == ROW_TERMINAL) {
      T lam[2][3] = {{0, 0, 0}, {0, 0, 0}};
      T qpsi[2] = {0, 0};
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int xi = x0 + i;
        T Bex[3] = {0, 0, 0};
        exchange_node(P, i, cx, cy, Bex);
        if (I.objective == 1) {
          const T V = (T)I.V, sc = (T)I.escale;
          const T pi = P.p[i];
          const T mdb = dot3(P.y[i], Bd[i]);
          vsum += -0.5 * (double)V * (double)Ms * (double)pi * (double)mdb;
          const T hh[4] = {(T)I.ihx2, (T)I.ihx2, (T)I.ihy2, (T)I.ihy2};
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            if (!P.ok[i][d]) continue;
            const T pj = P.pn[i][d];
            T dm2 = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const T dd = P.yn[i][d][c] - P.y[i][c];
              dm2 += dd * dd;
            }
            const T sp = pi + pj;
            const T Aij = sp > (T)0 ? (T)2 * (T)I.A * pi * pj / sp : (T)0;
            vsum += 0.5 * (double)Aij * (double)V * (double)dm2 * (double)hh[d];
            if (sp > (T)0) qpsi[i] += (T)2 * (T)I.A * pj * pj / (sp * sp) * V * dm2 * hh[d] * sc;
          }
          qpsi[i] += -V * Ms * mdb * sc;
          const double meanpsi = a.psisum[tile.inst] / (double)nodes;
          qpsi[i] += (T)(2.0 * I.penalty_w * (meanpsi - I.area_target) / (double)nodes);
#pragma unroll
          for (int c = 0; c < 3; ++c) lam[i][c] = -V * Ms * pi * (Bd[i][c] + Bex[c]) * sc;
        } else if (a.nsteps >= a.n_from) {
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            if (!in_box(I.boxes[b], xi, y)) continue;
            const T vv = P.y[i][I.comp];
            lam[i][I.comp] += (T)I.wbox[b] * (I.power == 2 ? (T)2 * vv : (T)1);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) st2(a.lam + off3 + c * nodes + n0, lam[0][c], lam[1][c]);
      st2(a.psib + I.node_off + n0, qpsi[0], qpsi[1]);
      st2(a.psic + I.node_off + n0, (T)0, (T)0);
      continue;
    }
    T B[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int xi = x0 + i;
#pragma unroll
      for (int c = 0; c < 3; ++c) B[i][c] = Bd[i][c];
      exchange_node(P, i, cx, cy, B[i]);
      if (kan != (T)0) {
        const T d = dot3(P.y[i], ku);
#pragma unroll
        for (int c = 0; c < 3; ++c) B[i][c] += kan * d * ku[c];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) B[i][c] += (T)I.B_bias[c];
      if (in_box(I.src, xi, y)) {
#pragma unroll
        for (int c = 0; c < 3; ++c) B[i][c] += rf * (T)I.rf_dir[c];
      }
    }
    if (MODE == ROW_FIELD) {
#pragma unroll
      for (int c = 0; c < 3; ++c) st2(a.Bout + off3 + c * nodes + n0, B[0][c], B[1][c]);
      continue;
    }
    // ROW_STAGE: LL right-hand side and RK4 stage combine
    T k[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i) llg_rhs(P.y[i], B[i], alpha_at<T>(I, x0 + i, y), k[i]);
    if (a.Bout)
#pragma unroll
      for (int c = 0; c < 3; ++c) st2(a.Bout + off3 + c * nodes + n0, B[0][c], B[1][c]);
    T yn[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = off3 + c * nodes + n0;
      T m0, m1;
      ld2(a.m + id, m0, m1);
      if (s == 1) {
        st2(a.acc + id, k[0][c], k[1][c]);
        yn[0][c] = m0 + (T)0.5 * dt * k[0][c];
        yn[1][c] = m1 + (T)0.5 * dt * k[1][c];
      } else if (s == 2 || s == 3) {
        const T h = (s == 2) ? (T)0.5 * dt : dt;
        T a0, a1;
        ld2(a.acc + id, a0, a1);
        st2(a.acc + id, a0 + (T)2 * k[0][c], a1 + (T)2 * k[1][c]);
        yn[0][c] = m0 + h * k[0][c];
        yn[1][c] = m1 + h * k[1][c];
      } else {
        T a0, a1;
        ld2(a.acc + id, a0, a1);
        yn[0][c] = m0 + dt / (T)6 * (a0 + k[0][c]);
        yn[1][c] = m1 + dt / (T)6 * (a1 + k[1][c]);
        st2(a.mout + id, yn[0][c], yn[1][c]);
        if (a.ckpt) st2(a.ckpt + id, yn[0][c], yn[1][c]);
      }
      if (s < 4) st2(a.Yout + id, yn[0][c], yn[1][c]);
      v[c][q] = mk<C>(Ms * P.p[0] * yn[0][c], Ms * P.p[1] * yn[1][c]);
    }
    if (objective_step) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          if (!in_box(I.boxes[b], x0 + i, y)) continue;
          const T vv = yn[i][I.comp];
          vsum += I.wbox[b] * (double)(I.power == 2 ? vv * vv : vv);
        }
    }
  }
  if (MODE == ROW_TERMINAL) {
    if (I.objective == 1) {
      const double tot = block_sum(vsum, red);
      if (threadIdx.x == 0) atomicAdd(a.jterm + tile.inst, tot * I.escale);
    }
    return;
  }
  if (objective_step) {
    bool touches = false;
    for (int b = 0; b < 2; ++b)
      touches |= (I.wbox[b] != 0.0) && I.boxes[b][2] < tile.y0 + tile.nrows && I.boxes[b][3] > tile.y0;
    if (touches) {
      const double tot = block_sum(vsum, red);
      if (threadIdx.x == 0) atomicAdd(a.slots + I.slot_off + n + 1, tot);
    }
  }
  if (MODE == ROW_FIELD) return;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 4; q < 8; ++q) v[c][q] = mk<C>((T)0, (T)0);
  row_forward<T, L>(v, row, active, sm, t, a.tw);
}

// ---------------------------------------------------------------------------
// forward RK4 stage with its inputs staged by bulk asynchronous copies.
//
// At entry one thread issues cp.async.bulk copies of the tile's packed field
// spectrum (barrier 0) and of the rows the stencil and the stage combine
// read: Y_s with one halo row on each side, psi with the same halo, m_n and
// the RK accumulator (barrier 1).  The inverse row FFTs run while the node
// data is in flight.  Shared memory: [exchange / spectrum staging]
// [Y halo 3 x (R+2) rows][psi halo (R+2) rows][m 3 x R rows][acc 3 x R rows].
// ---------------------------------------------------------------------------

template <typename T>
__host__ __device__ constexpr size_t stage_smem_bytes(int L, int nx) {
  return (size_t)rows_per_tile(L) * 3 * rf_padded_len(L) * sizeof(cplx<T>) +
         (size_t)(10 * rows_per_tile(L) + 8) * nx * sizeof(T);
}

// Neighbour data of the pair at (x0, row rr of the staged halo arrays).
template <typename T>
__device__ __forceinline__ void gather_pair_smem(const T* sF, int cstride, const T* sP, int nx, int ny, int x0,
                                                 int y, int rr, PairNbr<T>& q) {
  const bool has_l = x0 > 0, has_r = x0 + 2 < nx, has_u = y + 1 < ny, has_d = y > 0;
  const int o = rr * nx + x0;
  ld2(sP + o, q.p[0], q.p[1]);
  T pu0 = 0, pu1 = 0, pd0 = 0, pd1 = 0;
  if (has_u) ld2(sP + o + nx, pu0, pu1);
  if (has_d) ld2(sP + o - nx, pd0, pd1);
  const T pl = has_l ? sP[o - 1] : (T)0;
  const T pr = has_r ? sP[o + 2] : (T)0;
  q.pn[0][0] = q.p[1]; q.pn[0][1] = pl; q.pn[0][2] = pu0; q.pn[0][3] = pd0;
  q.pn[1][0] = pr;     q.pn[1][1] = q.p[0]; q.pn[1][2] = pu1; q.pn[1][3] = pd1;
  q.ok[0][0] = true;  q.ok[0][1] = has_l; q.ok[0][2] = has_u; q.ok[0][3] = has_d;
  q.ok[1][0] = has_r; q.ok[1][1] = true;  q.ok[1][2] = has_u; q.ok[1][3] = has_d;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T* F = sF + c * cstride + o;
    ld2(F, q.y[0][c], q.y[1][c]);
    T u0 = 0, u1 = 0, d0 = 0, d1 = 0;
    if (has_u) ld2(F + nx, u0, u1);
    if (has_d) ld2(F - nx, d0, d1);
    const T l = has_l ? F[-1] : (T)0;
    const T r = has_r ? F[2] : (T)0;
    q.yn[0][0][c] = q.y[1][c]; q.yn[0][1][c] = l; q.yn[0][2][c] = u0; q.yn[0][3][c] = d0;
    q.yn[1][0][c] = r;         q.yn[1][1][c] = q.y[0][c]; q.yn[1][2][c] = u1; q.yn[1][3][c] = d1;
  }
}

template <typename T, int L>
__device__ __forceinline__ void stage_body(const RowArgs<T>& a, const DevInst& I, const RowTile& tile,
                                           unsigned char* smem_raw, uint64_t* bars, double* red, T rf) {
  using C = cplx<T>;
  constexpr int TT = L / 8;
  constexpr int SP = rf_padded_len(L);
  constexpr int RM = rows_per_tile(L);
  const int tid = threadIdx.x;
  const int rl = tid / TT, t = tid - rl * TT;
  const int nr = tile.nrows;
  const bool active = rl < nr;
  const int nx = I.nx, ny = I.ny, y0 = tile.y0;
  const int y = y0 + (active ? rl : 0);
  const long long nodes = I.nodes;
  C* sx = reinterpret_cast<C*>(smem_raw);
  T* sY = reinterpret_cast<T*>(sx + RM * 3 * SP);
  T* sP = sY + 3 * (RM + 2) * nx;
  T* sM = sP + (RM + 2) * nx;
  T* sA = sM + 3 * RM * nx;
  const long long off3 = 3 * I.node_off;
  C* row0 = a.spec + I.spec_off + (long long)y0 * 3 * L;
  const int s = a.stage;
  const long long n = (a.step_base ? *a.step_base : 0) + a.local_step;
  const int ylo = max(0, y0 - 1), yhi = min(ny, y0 + nr + 1);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned sb = (unsigned)(nr * 3 * L * sizeof(C));
    mbar_arrive_expect(&bars[0], sb);
    bulk_load(sx, row0, sb, &bars[0]);
    const unsigned hb = (unsigned)((yhi - ylo) * nx * sizeof(T));
    const unsigned rb = (unsigned)(nr * nx * sizeof(T));
    const bool need_acc = s > 1;
    mbar_arrive_expect(&bars[1], 4 * hb + 3 * rb + (need_acc ? 3 * rb : 0));
    const int r0 = ylo - y0 + 1;
    for (int c = 0; c < 3; ++c)
      bulk_load(sY + (c * (RM + 2) + r0) * nx, a.Yin + off3 + c * nodes + (long long)ylo * nx, hb, &bars[1]);
    bulk_load(sP + r0 * nx, a.psi + I.node_off + (long long)ylo * nx, hb, &bars[1]);
    for (int c = 0; c < 3; ++c)
      bulk_load(sM + c * RM * nx, a.m + off3 + c * nodes + (long long)y0 * nx, rb, &bars[1]);
    if (need_acc)
      for (int c = 0; c < 3; ++c)
        bulk_load(sA + c * RM * nx, a.acc + off3 + c * nodes + (long long)y0 * nx, rb, &bars[1]);
  }
  // inverse row FFTs of the field spectra while the node data arrives
  mbar_wait(&bars[0], 0, a.err);
  C v[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < 8; ++q)
      v[c][q] = active ? unpack_one(sx + (rl * 3 + c) * L, t + TT * q, L, a.tw) : mk<C>((T)0, (T)0);
  __syncthreads();
  regfft<C, L, 1, 3>(v, sx + rl * 3 * SP, SP, 1, t, a.tw);
  mbar_wait(&bars[1], 0, a.err);

  const T Ms = (T)I.Ms, cx = (T)I.cex_x, cy = (T)I.cex_y, kan = (T)I.kan;
  const T ku[3] = {(T)I.ku[0], (T)I.ku[1], (T)I.ku[2]};
  const T dt = (T)a.dt;
  double vsum = 0.0;
  const bool objective_step = s == 4 && a.slots != nullptr && I.objective == 0 && (n + 1) >= a.n_from;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int x0 = 2 * (t + TT * q);
    if (!active || x0 >= nx) {
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][q] = mk<C>((T)0, (T)0);
      continue;
    }
    PairNbr<T> P;
    gather_pair_smem(sY, (RM + 2) * nx, sP, nx, ny, x0, y, rl + 1, P);
    T B[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
      for (int c = 0; c < 3; ++c) B[i][c] = (i == 0) ? v[c][q].x : v[c][q].y;
      exchange_node(P, i, cx, cy, B[i]);
      if (kan != (T)0) {
        const T d = dot3(P.y[i], ku);
#pragma unroll
        for (int c = 0; c < 3; ++c) B[i][c] += kan * d * ku[c];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) B[i][c] += (T)I.B_bias[c];
      if (in_box(I.src, x0 + i, y)) {
#pragma unroll
        for (int c = 0; c < 3; ++c) B[i][c] += rf * (T)I.rf_dir[c];
      }
    }
    T k[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i) llg_rhs(P.y[i], B[i], alpha_at<T>(I, x0 + i, y), k[i]);
    const long long n0 = (long long)y * nx + x0;
    if (a.Bout)
#pragma unroll
      for (int c = 0; c < 3; ++c) st2(a.Bout + off3 + c * nodes + n0, B[0][c], B[1][c]);
    T yn[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = off3 + c * nodes + n0;
      const int so = (c * RM + rl) * nx + x0;
      T m0, m1;
      ld2(sM + so, m0, m1);
      if (s == 1) {
        st2(a.acc + id, k[0][c], k[1][c]);
        yn[0][c] = m0 + (T)0.5 * dt * k[0][c];
        yn[1][c] = m1 + (T)0.5 * dt * k[1][c];
      } else if (s == 2 || s == 3) {
        const T h = (s == 2) ? (T)0.5 * dt : dt;
        T a0, a1;
        ld2(sA + so, a0, a1);
        st2(a.acc + id, a0 + (T)2 * k[0][c], a1 + (T)2 * k[1][c]);
        yn[0][c] = m0 + h * k[0][c];
        yn[1][c] = m1 + h * k[1][c];
      } else {
        T a0, a1;
        ld2(sA + so, a0, a1);
        yn[0][c] = m0 + dt / (T)6 * (a0 + k[0][c]);
        yn[1][c] = m1 + dt / (T)6 * (a1 + k[1][c]);
        st2(a.mout + id, yn[0][c], yn[1][c]);
        if (a.ckpt) st2(a.ckpt + id, yn[0][c], yn[1][c]);
      }
      if (s < 4) st2(a.Yout + id, yn[0][c], yn[1][c]);
      v[c][q] = mk<C>(Ms * P.p[0] * yn[0][c], Ms * P.p[1] * yn[1][c]);
    }
    if (objective_step) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          if (!in_box(I.boxes[b], x0 + i, y)) continue;
          const T vv = yn[i][I.comp];
          vsum += I.wbox[b] * (double)(I.power == 2 ? vv * vv : vv);
        }
    }
  }
  if (objective_step) {
    bool touches = false;
    for (int b = 0; b < 2; ++b)
      touches |= (I.wbox[b] != 0.0) && I.boxes[b][2] < y0 + nr && I.boxes[b][3] > y0;
    if (touches) {
      const double tot = block_sum(vsum, red);
      if (threadIdx.x == 0) atomicAdd(a.slots + I.slot_off + n + 1, tot);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 4; q < 8; ++q) v[c][q] = mk<C>((T)0, (T)0);
  row_forward<T, L>(v, a.spec + I.spec_off + (long long)y * 3 * L, active, sx + rl * 3 * SP, t, a.tw);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kRowThreads) rows_kernel(RowArgs<T> a) {
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
    } else {
      s_rf = 0.0;
    }
  }
  __syncthreads();
  C* sm = reinterpret_cast<C*>(smem_raw);
  const T rf = (T)s_rf;
  if (MODE == ROW_STAGE) {
    switch (sI.log2Lx) {
      case 3: stage_body<T, 8>(a, sI, tile, smem_raw, bars, red, rf); break;
      case 4: stage_body<T, 16>(a, sI, tile, smem_raw, bars, red, rf); break;
      case 5: stage_body<T, 32>(a, sI, tile, smem_raw, bars, red, rf); break;
      case 6: stage_body<T, 64>(a, sI, tile, smem_raw, bars, red, rf); break;
      case 7: stage_body<T, 128>(a, sI, tile, smem_raw, bars, red, rf); break;
      case 8: stage_body<T, 256>(a, sI, tile, smem_raw, bars, red, rf); break;
      case 9: stage_body<T, 512>(a, sI, tile, smem_raw, bars, red, rf); break;
      case 10: stage_body<T, 1024>(a, sI, tile, smem_raw, bars, red, rf); break;
      default: break;
    }
    return;
  }
  switch (sI.log2Lx) {
    case 3: rows_body<T, 8, MODE>(a, sI, tile, sm, red, rf); break;
    case 4: rows_body<T, 16, MODE>(a, sI, tile, sm, red, rf); break;
    case 5: rows_body<T, 32, MODE>(a, sI, tile, sm, red, rf); break;
    case 6: rows_body<T, 64, MODE>(a, sI, tile, sm, red, rf); break;
    case 7: rows_body<T, 128, MODE>(a, sI, tile, sm, red, rf); break;
    case 8: rows_body<T, 256, MODE>(a, sI, tile, sm, red, rf); break;
    case 9: rows_body<T, 512, MODE>(a, sI, tile, sm, red, rf); break;
    case 10: rows_body<T, 1024, MODE>(a, sI, tile, sm, red, rf); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// adjoint stage
// ---------------------------------------------------------------------------

template <typename T, int L>
__device__ __forceinline__ void adj_body(const AdjArgs<T>& a, const DevInst& I, const RowTile& tile,
                                         cplx<T>* smem) {
  using C = cplx<T>;
  constexpr int TT = L / 8;
  const int tid = threadIdx.x;
  const int rl = tid / TT, t = tid - rl * TT;
  const bool active = rl < tile.nrows;
  const int nx = I.nx, ny = I.ny;
  const int y = tile.y0 + (active ? rl : 0);
  const long long nodes = I.nodes;
  C* sm = smem + rl * 3 * rf_padded_len(L);
  C* row = a.spec + I.spec_off + (long long)y * 3 * L;
  const long long n = (a.step_base ? *a.step_base : 0) + a.local_step;
  const int s = a.stage;
  const long long off3 = 3 * I.node_off;
  const T* __restrict__ ps = a.psi + I.node_off;
  const T Ms = (T)I.Ms, cx = (T)I.cex_x, cy = (T)I.cex_y, kan = (T)I.kan;
  const T ku[3] = {(T)I.ku[0], (T)I.ku[1], (T)I.ku[2]};
  const T dt = (T)a.dt;
  T ca = 0, cb = 0;   // u_{s-1} = ca lambda + cb g_s
  if (s == 4) { ca = dt / (T)3; cb = dt; }
  else if (s == 3) { ca = dt / (T)3; cb = (T)0.5 * dt; }
  else if (s == 2) { ca = dt / (T)6; cb = (T)0.5 * dt; }
  const bool emit = a.seed_only || s > 1 || a.seed_next;

  C v[3][8];
  if (!a.seed_only) row_inverse<T, L>(v, row, active, sm, t, a.tw);

#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int x0 = 2 * (t + TT * q);
    if (!active || x0 >= nx) {
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][q] = mk<C>((T)0, (T)0);
      continue;
    }
    const long long n0 = (long long)y * nx + x0;
    T lam[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) ld2(a.lam + off3 + c * nodes + n0, lam[0][c], lam[1][c]);
    T u[2][3];
    if (a.seed_only) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) u[i][c] = dt / (T)6 * lam[i][c];
    } else {
      PairNbr<T> Py, Pb;   // stage input Y_s and field cotangent Bbar_s around the pair
      gather_pair(a.Ys + off3, ps, nodes, nx, ny, x0, y, Py);
      gather_pair(a.Bbar + off3, ps, nodes, nx, ny, x0, y, Pb);
      T g[2][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) ld2(a.gpart + off3 + c * nodes + n0, g[0][c], g[1][c]);
      T qpsi[2] = {0, 0};
      const T cc[4] = {cx, cx, cy, cy};
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const T pi = Py.p[i];
        // exchange transpose (gather form) and its psi derivative
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          if (!Py.ok[i][d]) continue;
          const T pj = Py.pn[i][d];
          const T wij = edge_weight(pi, pj), wji = edge_weight(pj, pi);
          T eij = 0, eji = 0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            g[i][c] += cc[d] * (wji * Pb.yn[i][d][c] - wij * Pb.y[i][c]);
            eij += Pb.y[i][c] * (Py.yn[i][d][c] - Py.y[i][c]);
            eji += Pb.yn[i][d][c] * (Py.y[i][c] - Py.yn[i][d][c]);
          }
          const T sp = pi + pj;
          if (sp > (T)0) qpsi[i] += cc[d] * (T)2 * pj / (sp * sp) * (eji - eij);
        }
        // demag transpose Ms psi_i (N * Bbar)_i and its psi derivative
        const T D[3] = {i == 0 ? v[0][q].x : v[0][q].y, i == 0 ? v[1][q].x : v[1][q].y,
                        i == 0 ? v[2][q].x : v[2][q].y};
#pragma unroll
        for (int c = 0; c < 3; ++c) g[i][c] += Ms * pi * D[c];
        qpsi[i] += Ms * dot3(Py.y[i], D);
      }
      {
        T s0, s1, c0, c1;
        ld2(a.psib + I.node_off + n0, s0, s1);
        ld2(a.psic + I.node_off + n0, c0, c1);
        kahan_add(s0, c0, qpsi[0]);
        kahan_add(s1, c1, qpsi[1]);
        st2(a.psib + I.node_off + n0, s0, s1);
        st2(a.psic + I.node_off + n0, c0, c1);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long id = off3 + c * nodes + n0;
        if (s == 4) {
          st2(a.G + id, g[0][c], g[1][c]);
        } else if (s > 1) {
          T g0, g1;
          ld2(a.G + id, g0, g1);
          st2(a.G + id, g0 + g[0][c], g1 + g[1][c]);
        } else {
          T g0, g1;
          ld2(a.G + id, g0, g1);
          lam[0][c] += g0 + g[0][c];
          lam[1][c] += g1 + g[1][c];
        }
      }
      if (s == 1) {
        if (I.objective == 0 && n >= a.n_from) {
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
              if (!in_box(I.boxes[b], x0 + i, y)) continue;
              const T vv = Py.y[i][I.comp];
              lam[i][I.comp] += (T)I.wbox[b] * (I.power == 2 ? (T)2 * vv : (T)1);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) st2(a.lam + off3 + c * nodes + n0, lam[0][c], lam[1][c]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) u[i][c] = (s > 1) ? ca * lam[i][c] + cb * g[i][c] : dt / (T)6 * lam[i][c];
    }
    if (!emit) continue;
    T yp[2][3], bp[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ld2(a.Yprev + off3 + c * nodes + n0, yp[0][c], yp[1][c]);
      ld2(a.Bprev + off3 + c * nodes + n0, bp[0][c], bp[1][c]);
    }
    T bbar[2][3], gl[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      rhs_vjp(u[i], yp[i], bp[i], alpha_at<T>(I, x0 + i, y), bbar[i], gl[i]);
      if (kan != (T)0) {
        const T d = dot3(bbar[i], ku);
#pragma unroll
        for (int c = 0; c < 3; ++c) gl[i][c] += kan * d * ku[c];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long id = off3 + c * nodes + n0;
      st2(a.BbarOut + id, bbar[0][c], bbar[1][c]);
      st2(a.gpart + id, gl[0][c], gl[1][c]);
      v[c][q] = mk<C>(bbar[0][c], bbar[1][c]);
    }
  }
  if (!emit) return;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 4; q < 8; ++q) v[c][q] = mk<C>((T)0, (T)0);
  row_forward<T, L>(v, row, active, sm, t, a.tw);
}

template <typename T>
__global__ void __launch_bounds__(kAdjThreads) adj_kernel(AdjArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevInst sI;
  const RowTile tile = a.tiles[blockIdx.x];
  load_inst(sI, a.inst + tile.inst);
  __syncthreads();
  C* sm = reinterpret_cast<C*>(smem_raw);
  switch (sI.log2Lx) {
    case 3: adj_body<T, 8>(a, sI, tile, sm); break;
    case 4: adj_body<T, 16>(a, sI, tile, sm); break;
    case 5: adj_body<T, 32>(a, sI, tile, sm); break;
    case 6: adj_body<T, 64>(a, sI, tile, sm); break;
    case 7: adj_body<T, 128>(a, sI, tile, sm); break;
    case 8: adj_body<T, 256>(a, sI, tile, sm); break;
    case 9: adj_body<T, 512>(a, sI, tile, sm); break;
    case 10: adj_body<T, 1024>(a, sI, tile, sm); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// elementwise kernels (one CTA per row tile)
// ---------------------------------------------------------------------------

template <typename T>
__global__ void material_kernel(const DevInst* inst, const RowTile* tiles, const T* phi, T* psi, T* dpsi,
                                double* psisum) {
  __shared__ double red[32];
  const RowTile tile = tiles[blockIdx.x];
  const DevInst& I = inst[tile.inst];
  const long long base = I.node_off + (long long)tile.y0 * I.nx;
  const int cnt = tile.nrows * I.nx;
  double acc = 0.0;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const double ph = (double)phi[base + e];
    const double p = 1.0 / (1.0 + exp(-I.sigmoid_a * ph));   // Eq. 4
    psi[base + e] = (T)p;
    dpsi[base + e] = (T)(I.sigmoid_a * p * (1.0 - p));
    acc += p;
  }
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(psisum + tile.inst, tot);
}

template <typename T>
__global__ void grad_finish_kernel(const DevInst* inst, const RowTile* tiles, const T* dpsi, const T* psib,
                                   const T* psic, T* out) {
  const RowTile tile = tiles[blockIdx.x];
  const DevInst& I = inst[tile.inst];
  const long long base = I.node_off + (long long)tile.y0 * I.nx;
  const int cnt = tile.nrows * I.nx;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const double g = ((double)psib[base + e] - (double)psic[base + e]) * (double)dpsi[base + e];
    out[base + e] = (T)g;
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
  const long long base = I.node_off + (long long)tile.y0 * I.nx;
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
  const long long base = I.node_off + (long long)tile.y0 * I.nx;
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
void launch_rows_mode(const RowArgs<T>& a, int ntiles, size_t smem, cudaStream_t st) {
  rows_kernel<T, MODE><<<ntiles, kRowThreads, smem, st>>>(a);
}
template <typename T, int MODE>
void smem_rows_mode(size_t smem) {
  cudaFuncSetAttribute(rows_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <typename T>
void launch_cols(const ColArgs<T>& a, int ntiles, size_t smem, cudaStream_t st) {
  cols_kernel<T><<<ntiles, kColThreads, smem, st>>>(a);
}
template <typename T>
void smem_cols(size_t smem) {
  cudaFuncSetAttribute(cols_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <typename T>
void launch_adj(const AdjArgs<T>& a, int ntiles, size_t smem, cudaStream_t st) {
  adj_kernel<T><<<ntiles, kAdjThreads, smem, st>>>(a);
}
template <typename T>
void smem_adj(size_t smem) {
  cudaFuncSetAttribute(adj_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <typename T>
void launch_material_tiles(const DevInst* inst, const RowTile* tiles, int ntiles, const T* phi, T* psi,
                           T* dpsi, double* psisum, cudaStream_t st) {
  material_kernel<T><<<ntiles, 256, 0, st>>>(inst, tiles, phi, psi, dpsi, psisum);
}
template <typename T>
void launch_grad_finish_tiles(const DevInst* inst, const RowTile* tiles, int ntiles, const T* dpsi,
                              const T* psib, const T* psic, T* out, cudaStream_t st) {
  grad_finish_kernel<T><<<ntiles, 256, 0, st>>>(inst, tiles, dpsi, psib, psic, out);
}
template <typename T>
void launch_levelset_tiles(const DevInst* inst, const RowTile* tiles, int ntiles, T* phi, const T* grad,
                           const unsigned char* mask, double lr, unsigned int* maxbits, cudaStream_t st) {
  levelset_update_kernel<T><<<ntiles, 256, 0, st>>>(inst, tiles, phi, grad, mask, (T)lr, maxbits);
  levelset_scale_kernel<T><<<ntiles, 256, 0, st>>>(inst, tiles, phi, mask, maxbits);
}

}  // namespace llg
