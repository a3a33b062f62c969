// Hot-path kernels of the LLG forward pass and its discrete adjoint.
//
// One RK4 stage is two launches over every instance of the batch:
//   cols_kernel  column pass of the demag convolution: forward FFT along y
//                of the zero-padded row spectra, the pointwise product with
//                the tensor spectrum, inverse FFT along y (in shared memory);
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
#include <climits>

#include "fft.cuh"
#include "kernels.cuh"

namespace llg {

constexpr int kRowThreads = 256;
constexpr int kColThreads = 256;
constexpr int kAdjThreads = 256;

int rows_threads() { return kRowThreads; }
int cols_threads() { return kColThreads; }
int adj_threads() { return kAdjThreads; }

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

// Block-wide sum of a double; result valid in thread 0.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

template <typename T>
__device__ __forceinline__ void kahan_add(T& sum, T& comp, T v) {
  const T y = v - comp;
  const T t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// inverse packing: Z[k] = (X_k + conj X_{Lx-k}) + i W_P^{-k} (X_k - conj X_{Lx-k})
template <typename C>
__device__ __forceinline__ void unpack_rows(const C* __restrict__ X, C* __restrict__ Z, int nseq, int Lx,
                                            int lg, const C* __restrict__ tw) {
  const int tstride = kTwiddleN >> (lg + 1);   // W_P with P = 2 Lx
  for (int e = threadIdx.x; e < nseq * Lx; e += blockDim.x) {
    const int q = e >> lg, k = e & (Lx - 1);
    const C xk = X[e];
    C z;
    if (k == 0) {
      z = mk<C>(xk.x + xk.y, xk.x - xk.y);
    } else {
      const C xm = cconj(X[(q << lg) + Lx - k]);
      C w = tw[k * tstride];
      w.y = -w.y;                                   // W_P^{-k}
      z = cadd(cadd(xk, xm), mul_pi(cmul(w, csub(xk, xm))));
    }
    Z[e] = z;
  }
}

// forward packing of Z = FFT(x[2j] + i x[2j+1]) into the packed row spectrum:
// X[k] = (Z_k + conj Z_{Lx-k})/2 - i W_P^k (Z_k - conj Z_{Lx-k})/2, X[0] = (Re+Im, Re-Im)
template <typename C>
__device__ __forceinline__ void pack_rows(const C* __restrict__ Z, C* __restrict__ out, int nseq, int Lx,
                                          int lg, const C* __restrict__ tw) {
  using R = decltype(C::x);
  const int tstride = kTwiddleN >> (lg + 1);
  for (int e = threadIdx.x; e < nseq * Lx; e += blockDim.x) {
    const int q = e >> lg, k = e & (Lx - 1);
    const C zk = Z[e];
    C x;
    if (k == 0) {
      x = mk<C>(zk.x + zk.y, zk.x - zk.y);
    } else {
      const C zm = cconj(Z[(q << lg) + Lx - k]);
      const C w = tw[k * tstride];
      const C even = cadd(zk, zm);
      const C odd = mul_mi(cmul(w, csub(zk, zm)));
      x = cscale(cadd(even, odd), (R)0.5);
    }
    out[e] = x;
  }
}

// ---------------------------------------------------------------------------
// column pass: FFT_y, product with the tensor spectrum, inverse FFT_y
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void load_tensor(const T* tab, long long idx, T n[4]) {
  const T* p = tab + idx * 4;
  n[0] = p[0]; n[1] = p[1]; n[2] = p[2]; n[3] = p[3];
}

template <typename T>
__global__ void __launch_bounds__(kColThreads) cols_kernel(ColArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ColTile tile = a.tiles[blockIdx.x];
  __shared__ DevInst sI;
  if (threadIdx.x == 0) sI = a.inst[tile.inst];
  __syncthreads();
  const DevInst& I = sI;
  const int ny = I.ny, Lx = I.Lx, Py = I.Py, lgy = I.log2Py;
  const int TX = tile.ncols, nseq = 3 * TX;
  const int ss = Py + 1;                         // padded sequence stride
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + (size_t)nseq * ss;
  C* spec = a.spec + I.spec_off;
  const int tid = threadIdx.x, nt = blockDim.x;

  // load the ny nonzero rows of the TX columns, zero-fill the padding
  for (int e = tid; e < ny * nseq; e += nt) {
    const int y = e / nseq, rem = e - y * nseq;
    const int c = rem / TX, col = rem - c * TX;
    bufA[(c * TX + col) * ss + y] = spec[((long long)y * 3 + c) * Lx + tile.kx0 + col];
  }
  const int npad = Py - ny;
  for (int e = tid; e < npad * nseq; e += nt) {
    const int q = e / npad, y = ny + (e - q * npad);
    bufA[q * ss + y] = mk<C>((T)0, (T)0);
  }
  __syncthreads();
  C* r = fft_batch<C, -1>(bufA, bufB, lgy, nseq, a.tw, ss);

  // product with the tensor spectrum (real, 4 components in 2D)
  const T* tab = a.tens + I.tens_off;
  const int nky = Py / 2 + 1;
  for (int e = tid; e < TX * Py; e += nt) {
    const int col = e / Py, ky = e - col * Py;
    const int kx = tile.kx0 + col;
    C* m0 = r + (0 * TX + col) * ss;
    C* m1 = r + (1 * TX + col) * ss;
    C* m2 = r + (2 * TX + col) * ss;
    if (kx != 0) {
      const bool lo = ky <= Py / 2;
      const int kyf = lo ? ky : Py - ky;
      T n[4];
      load_tensor(tab, (long long)kx * nky + kyf, n);
      const T nxy = lo ? n[3] : -n[3];
      const C mx = m0[ky], my = m1[ky], mz = m2[ky];
      m0[ky] = mk<C>(n[0] * mx.x + nxy * my.x, n[0] * mx.y + nxy * my.y);
      m1[ky] = mk<C>(nxy * mx.x + n[1] * my.x, nxy * mx.y + n[1] * my.y);
      m2[ky] = mk<C>(n[2] * mz.x, n[2] * mz.y);
    } else if (ky <= Py / 2) {
      // packed DC (kx = 0) and Nyquist (kx = Px/2) columns: separate them by
      // Hermitian symmetry in ky, apply each its own (diagonal) tensor, repack
      const int km = (Py - ky) & (Py - 1);
      T nd[4], nq[4];
      load_tensor(tab, (long long)0 * nky + ky, nd);
      load_tensor(tab, (long long)Lx * nky + ky, nq);
      C* mc[3] = {m0, m1, m2};
      for (int c = 0; c < 3; ++c) {
        const T p = (T)0.5 * (nd[c] + nq[c]), q = (T)0.5 * (nd[c] - nq[c]);
        const C va = mc[c][ky], vb = mc[c][km];
        mc[c][ky] = cadd(cscale(va, p), cscale(cconj(vb), q));
        if (km != ky) mc[c][km] = cadd(cscale(vb, p), cscale(cconj(va), q));
      }
    }
  }
  __syncthreads();
  C* r2 = fft_batch<C, 1>(r, r == bufA ? bufB : bufA, lgy, nseq, a.tw, ss);
  for (int e = tid; e < ny * nseq; e += nt) {
    const int y = e / nseq, rem = e - y * nseq;
    const int c = rem / TX, col = rem - c * TX;
    spec[((long long)y * 3 + c) * Lx + tile.kx0 + col] = r2[(c * TX + col) * ss + y];
  }
}

// ---------------------------------------------------------------------------
// row pass of the forward stage (and its variants)
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void exchange_at(const T* __restrict__ Y, const T* __restrict__ psi,
                                            long long nodes, int nx, int ny, int x, int y, long long node,
                                            const T yi[3], T pi, T cx, T cy, T B[3]) {
  const long long nb[4] = {node + 1, node - 1, node + nx, node - nx};
  const bool ok[4] = {x < nx - 1, x > 0, y < ny - 1, y > 0};
  const T cc[4] = {cx, cx, cy, cy};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    if (!ok[d]) continue;
    const long long j = nb[d];
    const T w = cc[d] * edge_weight(pi, psi[j]);
#pragma unroll
    for (int c = 0; c < 3; ++c) B[c] += w * (Y[c * nodes + j] - yi[c]);
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kRowThreads) rows_kernel(RowArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kRowThreads / 32];
  __shared__ double s_rf;
  const RowTile tile = a.tiles[blockIdx.x];
  __shared__ DevInst sI;
  if (threadIdx.x == 0) sI = a.inst[tile.inst];
  __syncthreads();
  const DevInst& I = sI;
  const int nx = I.nx, ny = I.ny, Lx = I.Lx, lg = I.log2Lx;
  const int R = tile.nrows, nseq = 3 * R;
  const long long nodes = I.nodes;
  const int tid = threadIdx.x, nt = blockDim.x;
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + (size_t)nseq * Lx;
  C* rows_g = a.spec + I.spec_off + (long long)tile.y0 * 3 * Lx;
  const long long n = (a.step_base ? *a.step_base : 0) + a.local_step;
  const int s = a.stage;

  T* Hd = nullptr;
  C* work = bufA;
  if (MODE != ROW_FFT_ONLY) {
    for (int e = tid; e < nseq * Lx; e += nt) bufA[e] = rows_g[e];
    __syncthreads();
    unpack_rows(bufA, bufB, nseq, Lx, lg, a.tw);
    __syncthreads();
    C* res = fft_batch<C, 1>(bufB, bufA, lg, nseq, a.tw);
    Hd = reinterpret_cast<T*>(res);
    work = (res == bufA) ? bufB : bufA;
  }
  if (tid == 0) {
    double t;
    if (MODE == ROW_FIELD) {
      t = a.t_field;
    } else {
      const double cs = (s == 1) ? 0.0 : (s == 4 ? 1.0 : 0.5);
      t = (double)n * a.dt + cs * a.dt;
    }
    s_rf = I.b_rf * sin(2.0 * M_PI * I.f_rf * t);
  }
  T* Mw = reinterpret_cast<T*>(work);
  if (MODE == ROW_FFT_ONLY || MODE == ROW_STAGE) {
    const int tail = 2 * Lx - nx;
    for (int e = tid; e < nseq * tail; e += nt) {
      const int q = e / tail;
      Mw[q * 2 * Lx + nx + (e - q * tail)] = (T)0;
    }
  }
  __syncthreads();

  const long long off3 = 3 * I.node_off;
  const T* __restrict__ Y = a.Yin + off3;
  const T* __restrict__ ps = a.psi + I.node_off;
  const T Ms = (T)I.Ms, cx = (T)I.cex_x, cy = (T)I.cex_y, kan = (T)I.kan;
  const T ku[3] = {(T)I.ku[0], (T)I.ku[1], (T)I.ku[2]};
  const T rf = (T)s_rf;
  double vsum = 0.0;
  const bool objective_step = (MODE == ROW_STAGE) && s == 4 && a.slots != nullptr &&
                              I.objective == 0 && (n + 1) >= a.n_from;

  for (int e = tid; e < R * nx; e += nt) {
    const int r = e / nx, x = e - r * nx, y = tile.y0 + r;
    const long long node = (long long)y * nx + x;
    const T yi[3] = {Y[node], Y[nodes + node], Y[2 * nodes + node]};
    const T pi = ps[node];
    if (MODE == ROW_FFT_ONLY) {
      for (int c = 0; c < 3; ++c) Mw[(r * 3 + c) * 2 * Lx + x] = Ms * pi * yi[c];
      continue;
    }
    T B[3] = {(T)0, (T)0, (T)0};
    T Bd[3];
    for (int c = 0; c < 3; ++c) Bd[c] = Hd[(r * 3 + c) * 2 * Lx + x];
    if (MODE == ROW_FIELD && a.demag_only) {
      for (int c = 0; c < 3; ++c) a.Bout[off3 + c * nodes + node] = Bd[c];
      continue;
    }
    exchange_at(Y, ps, nodes, nx, ny, x, y, node, yi, pi, cx, cy, B);
    if (MODE == ROW_TERMINAL) {
      // energies, lambda_N and explicit dJ/dpsi at m_N = Yin
      T lam[3] = {(T)0, (T)0, (T)0};
      T qpsi = (T)0;
      if (I.objective == 1) {
        const T V = (T)I.V, sc = (T)I.escale;
        const T mdb = dot3(yi, Bd);
        vsum += -0.5 * (double)V * (double)Ms * (double)pi * (double)mdb;
        // exchange energy, half of each edge here; dA_ij/dpsi_i terms
        const long long nb[4] = {node + 1, node - 1, node + nx, node - nx};
        const bool ok[4] = {x < nx - 1, x > 0, y < ny - 1, y > 0};
        const T hh[4] = {(T)I.ihx2, (T)I.ihx2, (T)I.ihy2, (T)I.ihy2};   // 1/h^2
        for (int d = 0; d < 4; ++d) {
          if (!ok[d]) continue;
          const long long j = nb[d];
          const T pj = ps[j];
          T dm2 = (T)0;
          for (int c = 0; c < 3; ++c) {
            const T dd = Y[c * nodes + j] - yi[c];
            dm2 += dd * dd;
          }
          const T sp = pi + pj;
          const T Aij = sp > (T)0 ? (T)2 * (T)I.A * pi * pj / sp : (T)0;
          vsum += 0.5 * (double)Aij * (double)V * (double)dm2 * (double)hh[d];
          if (sp > (T)0) qpsi += (T)2 * (T)I.A * pj * pj / (sp * sp) * V * dm2 * hh[d] * sc;
        }
        qpsi += -V * Ms * mdb * sc;
        const double meanpsi = a.psisum[tile.inst] / (double)nodes;
        qpsi += (T)(2.0 * I.penalty_w * (meanpsi - I.area_target) / (double)nodes);
        for (int c = 0; c < 3; ++c) lam[c] = -V * Ms * pi * (Bd[c] + B[c]) * sc;
      } else if (a.nsteps >= a.n_from) {
        for (int b = 0; b < 2; ++b) {
          if (!in_box(I.boxes[b], x, y)) continue;
          const T v = yi[I.comp];
          lam[I.comp] += (T)I.wbox[b] * (I.power == 2 ? (T)2 * v : (T)1);
        }
      }
      for (int c = 0; c < 3; ++c) a.lam[off3 + c * nodes + node] = lam[c];
      a.psib[I.node_off + node] = qpsi;
      a.psic[I.node_off + node] = (T)0;
      continue;
    }
    for (int c = 0; c < 3; ++c) B[c] += Bd[c];
    if (kan != (T)0) {
      const T d = dot3(yi, ku);
      for (int c = 0; c < 3; ++c) B[c] += kan * d * ku[c];
    }
    B[0] += (T)I.B_bias[0];
    B[1] += (T)I.B_bias[1];
    B[2] += (T)I.B_bias[2];
    if (in_box(I.src, x, y)) {
      B[0] += rf * (T)I.rf_dir[0];
      B[1] += rf * (T)I.rf_dir[1];
      B[2] += rf * (T)I.rf_dir[2];
    }
    if (MODE == ROW_FIELD) {
      for (int c = 0; c < 3; ++c) a.Bout[off3 + c * nodes + node] = B[c];
      continue;
    }
    // ROW_STAGE
    const T al = alpha_at<T>(I, x, y);
    T k[3];
    llg_rhs(yi, B, al, k);
    if (a.Bout)
      for (int c = 0; c < 3; ++c) a.Bout[off3 + c * nodes + node] = B[c];
    const T dt = (T)a.dt;
    T mn[3], yn[3];
    for (int c = 0; c < 3; ++c) mn[c] = a.m[off3 + c * nodes + node];
    if (s == 1) {
      for (int c = 0; c < 3; ++c) {
        a.acc[off3 + c * nodes + node] = k[c];
        yn[c] = mn[c] + (T)0.5 * dt * k[c];
      }
    } else if (s == 2 || s == 3) {
      const T h = (s == 2) ? (T)0.5 * dt : dt;
      for (int c = 0; c < 3; ++c) {
        const long long id = off3 + c * nodes + node;
        a.acc[id] = a.acc[id] + (T)2 * k[c];
        yn[c] = mn[c] + h * k[c];
      }
    } else {
      for (int c = 0; c < 3; ++c) {
        const long long id = off3 + c * nodes + node;
        yn[c] = mn[c] + dt / (T)6 * (a.acc[id] + k[c]);
        a.mout[id] = yn[c];
        if (a.ckpt) a.ckpt[id] = yn[c];
      }
      if (objective_step) {
        for (int b = 0; b < 2; ++b) {
          if (!in_box(I.boxes[b], x, y)) continue;
          const T v = yn[I.comp];
          vsum += I.wbox[b] * (double)(I.power == 2 ? v * v : v);
        }
      }
    }
    if (s < 4)
      for (int c = 0; c < 3; ++c) a.Yout[off3 + c * nodes + node] = yn[c];
    for (int c = 0; c < 3; ++c) Mw[(r * 3 + c) * 2 * Lx + x] = Ms * pi * yn[c];
  }

  if (MODE == ROW_TERMINAL) {
    if (I.objective == 1) {
      const double tot = block_sum(vsum, red);
      if (tid == 0) atomicAdd(a.jterm + tile.inst, tot * I.escale);
    }
    return;
  }
  if (objective_step) {
    bool touches = false;
    for (int b = 0; b < 2; ++b)
      touches |= (I.wbox[b] != 0.0) && I.boxes[b][2] < tile.y0 + R && I.boxes[b][3] > tile.y0;
    if (touches) {
      const double tot = block_sum(vsum, red);
      if (tid == 0) atomicAdd(a.slots + I.slot_off + n + 1, tot);
    }
  }
  if (MODE == ROW_FIELD) return;
  __syncthreads();
  C* other = (MODE == ROW_FFT_ONLY) ? bufB : reinterpret_cast<C*>(Hd);
  C* res = fft_batch<C, -1>(work, other, lg, nseq, a.tw);
  pack_rows(res, rows_g, nseq, Lx, lg, a.tw);
}

// ---------------------------------------------------------------------------
// adjoint stage
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kAdjThreads) adj_kernel(AdjArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RowTile tile = a.tiles[blockIdx.x];
  __shared__ DevInst sI;
  if (threadIdx.x == 0) sI = a.inst[tile.inst];
  __syncthreads();
  const DevInst& I = sI;
  const int nx = I.nx, ny = I.ny, Lx = I.Lx, lg = I.log2Lx;
  const int R = tile.nrows, nseq = 3 * R;
  const long long nodes = I.nodes;
  const int tid = threadIdx.x, nt = blockDim.x;
  C* bufA = reinterpret_cast<C*>(smem_raw);
  C* bufB = bufA + (size_t)nseq * Lx;
  C* rows_g = a.spec + I.spec_off + (long long)tile.y0 * 3 * Lx;
  const long long n = (a.step_base ? *a.step_base : 0) + a.local_step;
  const int s = a.stage;

  T* Dd = nullptr;
  C* work = bufA;
  if (!a.seed_only) {
    for (int e = tid; e < nseq * Lx; e += nt) bufA[e] = rows_g[e];
    __syncthreads();
    unpack_rows(bufA, bufB, nseq, Lx, lg, a.tw);
    __syncthreads();
    C* res = fft_batch<C, 1>(bufB, bufA, lg, nseq, a.tw);
    Dd = reinterpret_cast<T*>(res);
    work = (res == bufA) ? bufB : bufA;
  }
  const bool emit = a.seed_only || s > 1 || a.seed_next;
  T* Mw = reinterpret_cast<T*>(work);
  if (emit) {
    const int tail = 2 * Lx - nx;
    for (int e = tid; e < nseq * tail; e += nt) {
      const int q = e / tail;
      Mw[q * 2 * Lx + nx + (e - q * tail)] = (T)0;
    }
  }
  __syncthreads();

  const long long off3 = 3 * I.node_off;
  const T* __restrict__ ps = a.psi + I.node_off;
  const T Ms = (T)I.Ms, cx = (T)I.cex_x, cy = (T)I.cex_y, kan = (T)I.kan;
  const T ku[3] = {(T)I.ku[0], (T)I.ku[1], (T)I.ku[2]};
  const T dt = (T)a.dt;
  // u_{s-1} = ca * lambda + cb * g_s
  T ca = (T)0, cb = (T)0;
  if (s == 4) { ca = dt / (T)3; cb = dt; }
  else if (s == 3) { ca = dt / (T)3; cb = (T)0.5 * dt; }
  else if (s == 2) { ca = dt / (T)6; cb = (T)0.5 * dt; }

  for (int e = tid; e < R * nx; e += nt) {
    const int r = e / nx, x = e - r * nx, y = tile.y0 + r;
    const long long node = (long long)y * nx + x;
    T lam[3];
    for (int c = 0; c < 3; ++c) lam[c] = a.lam[off3 + c * nodes + node];
    T u[3];
    if (a.seed_only) {
      for (int c = 0; c < 3; ++c) u[c] = dt / (T)6 * lam[c];
    } else {
      const T* __restrict__ Ys = a.Ys + off3;
      const T* __restrict__ Bb = a.Bbar + off3;
      const T yi[3] = {Ys[node], Ys[nodes + node], Ys[2 * nodes + node]};
      const T bi[3] = {Bb[node], Bb[nodes + node], Bb[2 * nodes + node]};
      const T pi = ps[node];
      T g[3];
      for (int c = 0; c < 3; ++c) g[c] = a.gpart[off3 + c * nodes + node];
      T qpsi = (T)0;
      // exchange transpose (gather form) and its psi derivative
      const long long nb[4] = {node + 1, node - 1, node + nx, node - nx};
      const bool ok[4] = {x < nx - 1, x > 0, y < ny - 1, y > 0};
      const T cc[4] = {cx, cx, cy, cy};
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        if (!ok[d]) continue;
        const long long j = nb[d];
        const T pj = ps[j];
        const T wij = edge_weight(pi, pj), wji = edge_weight(pj, pi);
        T bj[3], yj[3];
        for (int c = 0; c < 3; ++c) {
          bj[c] = Bb[c * nodes + j];
          yj[c] = Ys[c * nodes + j];
        }
        T eij = (T)0, eji = (T)0;
        for (int c = 0; c < 3; ++c) {
          g[c] += cc[d] * (wji * bj[c] - wij * bi[c]);
          eij += bi[c] * (yj[c] - yi[c]);
          eji += bj[c] * (yi[c] - yj[c]);
        }
        const T sp = pi + pj;
        if (sp > (T)0) qpsi += cc[d] * (T)2 * pj / (sp * sp) * (eji - eij);
      }
      // demag transpose: Ms psi_i (N * Bbar)_i; its psi derivative Ms Y_i.(N * Bbar)_i
      T D[3];
      for (int c = 0; c < 3; ++c) D[c] = Dd[(r * 3 + c) * 2 * Lx + x];
      for (int c = 0; c < 3; ++c) g[c] += Ms * pi * D[c];
      qpsi += Ms * dot3(yi, D);
      {
        T sum = a.psib[I.node_off + node], comp = a.psic[I.node_off + node];
        kahan_add(sum, comp, qpsi);
        a.psib[I.node_off + node] = sum;
        a.psic[I.node_off + node] = comp;
      }
      if (s == 4) {
        for (int c = 0; c < 3; ++c) a.G[off3 + c * nodes + node] = g[c];
      } else if (s > 1) {
        for (int c = 0; c < 3; ++c) {
          const long long id = off3 + c * nodes + node;
          a.G[id] = a.G[id] + g[c];
        }
      } else {
        T nl[3];
        for (int c = 0; c < 3; ++c) nl[c] = lam[c] + a.G[off3 + c * nodes + node] + g[c];
        if (I.objective == 0 && n >= a.n_from) {
          for (int b = 0; b < 2; ++b) {
            if (!in_box(I.boxes[b], x, y)) continue;
            const T v = yi[I.comp];
            nl[I.comp] += (T)I.wbox[b] * (I.power == 2 ? (T)2 * v : (T)1);
          }
        }
        for (int c = 0; c < 3; ++c) {
          a.lam[off3 + c * nodes + node] = nl[c];
          lam[c] = nl[c];
        }
      }
      if (s > 1) {
        for (int c = 0; c < 3; ++c) u[c] = ca * lam[c] + cb * g[c];
      } else {
        for (int c = 0; c < 3; ++c) u[c] = dt / (T)6 * lam[c];
      }
    }
    if (!emit) continue;
    const T yp[3] = {a.Yprev[off3 + node], a.Yprev[off3 + nodes + node], a.Yprev[off3 + 2 * nodes + node]};
    const T bp[3] = {a.Bprev[off3 + node], a.Bprev[off3 + nodes + node], a.Bprev[off3 + 2 * nodes + node]};
    const T al = alpha_at<T>(I, x, y);
    T bbar[3], gl[3];
    rhs_vjp(u, yp, bp, al, bbar, gl);
    if (kan != (T)0) {
      const T d = dot3(bbar, ku);
      for (int c = 0; c < 3; ++c) gl[c] += kan * d * ku[c];
    }
    for (int c = 0; c < 3; ++c) {
      a.BbarOut[off3 + c * nodes + node] = bbar[c];
      a.gpart[off3 + c * nodes + node] = gl[c];
      Mw[(r * 3 + c) * 2 * Lx + x] = bbar[c];
    }
  }
  if (!emit) return;
  __syncthreads();
  C* other = a.seed_only ? bufB : reinterpret_cast<C*>(Dd);
  C* res = fft_batch<C, -1>(work, other, lg, nseq, a.tw);
  pack_rows(res, rows_g, nseq, Lx, lg, a.tw);
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

__global__ void set_step_kernel(long long* p, long long v) { *p = v; }

// J_i = Kahan sum of the per-step slots + terminal term + area penalty
__global__ void reduce_slots_kernel(const DevInst* inst, const double* slots, long long nslots,
                                    const double* jterm, const double* psisum, double* J) {
  __shared__ double red[32];
  const DevInst& I = inst[blockIdx.x];
  double sum = 0.0, comp = 0.0;
  for (long long k = threadIdx.x; k < nslots; k += blockDim.x) {
    const double y = slots[I.slot_off + k] - comp;
    const double t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  const double tot = block_sum(sum - comp, red);
  if (threadIdx.x == 0) {
    double j = tot + jterm[blockIdx.x];
    if (I.objective == 1) {
      const double f = psisum[blockIdx.x] / (double)I.nodes - I.area_target;
      j += I.penalty_w * f * f;
    }
    J[blockIdx.x] = j;
  }
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------

template <typename T>
void launch_rows(const RowArgs<T>& a, int mode, int ntiles, size_t smem, cudaStream_t st) {
  switch (mode) {
    case ROW_FFT_ONLY:
      rows_kernel<T, ROW_FFT_ONLY><<<ntiles, kRowThreads, smem, st>>>(a);
      break;
    case ROW_STAGE:
      rows_kernel<T, ROW_STAGE><<<ntiles, kRowThreads, smem, st>>>(a);
      break;
    case ROW_FIELD:
      rows_kernel<T, ROW_FIELD><<<ntiles, kRowThreads, smem, st>>>(a);
      break;
    default:
      rows_kernel<T, ROW_TERMINAL><<<ntiles, kRowThreads, smem, st>>>(a);
      break;
  }
}

template <typename T>
void launch_cols(const ColArgs<T>& a, int ntiles, size_t smem, cudaStream_t st) {
  cols_kernel<T><<<ntiles, kColThreads, smem, st>>>(a);
}

template <typename T>
void launch_adj(const AdjArgs<T>& a, int ntiles, size_t smem, cudaStream_t st) {
  adj_kernel<T><<<ntiles, kAdjThreads, smem, st>>>(a);
}

template <typename T>
void set_smem_limits(size_t smem) {
  cudaFuncSetAttribute(rows_kernel<T, ROW_FFT_ONLY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(rows_kernel<T, ROW_STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(rows_kernel<T, ROW_FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(rows_kernel<T, ROW_TERMINAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(cols_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

void launch_set_step(long long* step_base, long long v, cudaStream_t st) {
  set_step_kernel<<<1, 1, 0, st>>>(step_base, v);
}

void launch_reduce_slots(const DevInst* inst, int n_inst, const double* slots, long long nslots,
                         const double* jterm, const double* psisum, double* J, cudaStream_t st) {
  reduce_slots_kernel<<<n_inst, 256, 0, st>>>(inst, slots, nslots, jterm, psisum, J);
}

#define LLG_INSTANTIATE(T)                                                                              \
  template void launch_rows<T>(const RowArgs<T>&, int, int, size_t, cudaStream_t);                      \
  template void launch_cols<T>(const ColArgs<T>&, int, size_t, cudaStream_t);                            \
  template void launch_adj<T>(const AdjArgs<T>&, int, size_t, cudaStream_t);                             \
  template void set_smem_limits<T>(size_t);                                                              \
  template void launch_material_tiles<T>(const DevInst*, const RowTile*, int, const T*, T*, T*, double*, \
                                         cudaStream_t);                                                  \
  template void launch_grad_finish_tiles<T>(const DevInst*, const RowTile*, int, const T*, const T*,     \
                                            const T*, T*, cudaStream_t);                                 \
  template void launch_levelset_tiles<T>(const DevInst*, const RowTile*, int, T*, const T*,              \
                                         const unsigned char*, double, unsigned int*, cudaStream_t);

LLG_INSTANTIATE(float)
LLG_INSTANTIATE(double)

}  // namespace llg
