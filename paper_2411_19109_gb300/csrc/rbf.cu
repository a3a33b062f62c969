// RBF parameterisation of the level-set function (Eq. 2, Eq. 3 and the
// renormalisation of Phi to [-1, 1]), its chain rule dJ/ds, and Adam.
//
// Phi on the design box is built from nrx x nry multiquadric cones
//   g_k(x) = s_k - sqrt(|x - x_k|^2 + c^2)
// (centres at the centres of equal cells of the box, c = the centre
// spacing), combined by the p-norm F = ||g + dphi||_p - dphi with
// dphi = |min_{k, design} g_k| and renormalised, Phi = F / max_design |F|.
// The p-norm is evaluated as U (sum (u/U)^p)^(1/p), U = max u, which cannot
// overflow for p = 90.  dJ/ds is the exact derivative of this map, taken at
// the minimising (node, RBF) pair and the maximising node, the first in
// index order on ties (flat index j K + k for the pair, j for the node).
//
// Everything runs in FP64 (the map is small: design nodes x RBFs); Phi is
// written in the solver's precision.  Centre and node coordinates and g are
// formed with explicitly rounded operations so that the argmin / argmax do
// not depend on contraction.
#include <cmath>
#include <climits>
#include <cstdint>

#include "llg.h"

namespace {

constexpr int kThreads = 256;

struct Geo {
  int nx, box[4], nrx, nry, J, K;
  double dx, dy, hx, hy, c, p;
};

__device__ __forceinline__ double centre_x(const Geo& g, int k) {
  return __dadd_rn(__dmul_rn((double)g.box[0], g.dx), __dmul_rn((double)(k % g.nrx) + 0.5, g.hx));
}
__device__ __forceinline__ double centre_y(const Geo& g, int k) {
  return __dadd_rn(__dmul_rn((double)g.box[2], g.dy), __dmul_rn((double)(k / g.nrx) + 0.5, g.hy));
}
// design node j (row-major over the box) -> coordinates and grid index
__device__ __forceinline__ void node_of(const Geo& g, int j, double& x, double& y, long long& n) {
  const int bw = g.box[1] - g.box[0];
  const int ix = g.box[0] + j % bw, iy = g.box[2] + j / bw;
  x = __dmul_rn((double)ix, g.dx);
  y = __dmul_rn((double)iy, g.dy);
  n = (long long)iy * g.nx + ix;
}
__device__ __forceinline__ double cone(const Geo& g, const double* s, int k, double x, double y) {
  const double ex = __dsub_rn(x, centre_x(g, k)), ey = __dsub_rn(y, centre_y(g, k));
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(g.c, g.c));
  return __dsub_rn(s[k], sqrt(r2));
}

// (value, index) pairs: smaller value first, then smaller index
__device__ __forceinline__ bool better_min(double v, long long i, double bv, long long bi) {
  return v < bv || (v == bv && i < bi);
}
__device__ __forceinline__ bool better_max(double v, long long i, double bv, long long bi) {
  return v > bv || (v == bv && i < bi);
}

template <bool MAX>
__device__ void block_argext(double& v, long long& i) {
  __shared__ double sv[kThreads];
  __shared__ long long si[kThreads];
  sv[threadIdx.x] = v;
  si[threadIdx.x] = i;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double ov = sv[threadIdx.x + w];
      const long long oi = si[threadIdx.x + w];
      if (MAX ? better_max(ov, oi, sv[threadIdx.x], si[threadIdx.x])
              : better_min(ov, oi, sv[threadIdx.x], si[threadIdx.x])) {
        sv[threadIdx.x] = ov;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  v = sv[0];
  i = si[0];
  __syncthreads();
}

__device__ double block_sum(double v) {
  __shared__ double sv[kThreads];
  sv[threadIdx.x] = v;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sv[threadIdx.x] += sv[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sv[0];
  __syncthreads();
  return r;
}

// Workspace layout (doubles): F[J], norm[J], H[J], A[J], kmin_v[K], kmin_i[K]
// (as double), then scalars.
enum { S_M = 0, S_KM, S_DPHI, S_BIGM, S_JM, S_GF, S_DDPHI, S_COUNT };
struct Work {
  double *F, *norm, *H, *A, *kv, *ki, *sc;
};
Work carve(void* w, int J, int K) {
  double* d = static_cast<double*>(w);
  Work r;
  r.F = d;
  r.norm = r.F + J;
  r.H = r.norm + J;
  r.A = r.H + J;
  r.kv = r.A + J;
  r.ki = r.kv + K;
  r.sc = r.ki + K;
  return r;
}

// 1. per RBF k: min over design nodes of g_k (block per k)
__global__ void kmin_kernel(Geo g, const double* s, Work w) {
  const int k = blockIdx.x;
  double bv = INFINITY;
  long long bi = LLONG_MAX;
  for (int j = threadIdx.x; j < g.J; j += kThreads) {
    double x, y;
    long long n;
    node_of(g, j, x, y, n);
    const double v = cone(g, s, k, x, y);
    const long long fi = (long long)j * g.K + k;
    if (better_min(v, fi, bv, bi)) { bv = v; bi = fi; }
  }
  block_argext<false>(bv, bi);
  if (threadIdx.x == 0) {
    w.kv[k] = bv;
    w.ki[k] = (double)bi;
  }
}

// 2. the shift: min over k (single block)
__global__ void shift_kernel(Geo g, Work w) {
  double bv = INFINITY;
  long long bi = LLONG_MAX;
  for (int k = threadIdx.x; k < g.K; k += kThreads) {
    const double v = w.kv[k];
    const long long fi = (long long)w.ki[k];
    if (better_min(v, fi, bv, bi)) { bv = v; bi = fi; }
  }
  block_argext<false>(bv, bi);
  if (threadIdx.x == 0) {
    w.sc[S_M] = bv;
    w.sc[S_KM] = (double)(bi % g.K);
    w.sc[S_DPHI] = fabs(bv);
  }
}

// 3. per design node (block per node, threads over the RBFs): p-norm, F,
// and for the gradient A_j = sum_k W_jk.  Sums run in a fixed order (strided
// partial sums, then a tree), so results do not depend on scheduling.
__device__ double block_max(double v) {
  __shared__ double sv[kThreads];
  sv[threadIdx.x] = v;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sv[threadIdx.x] = fmax(sv[threadIdx.x], sv[threadIdx.x + w]);
    __syncthreads();
  }
  const double r = sv[0];
  __syncthreads();
  return r;
}

__global__ void norm_kernel(Geo g, const double* s, Work w, int want_a) {
  const int j = blockIdx.x;
  const double dphi = w.sc[S_DPHI];
  double x, y;
  long long n;
  node_of(g, j, x, y, n);
  double U = 0.0;
  for (int k = threadIdx.x; k < g.K; k += kThreads) U = fmax(U, cone(g, s, k, x, y) + dphi);
  U = block_max(U);
  double norm = 0.0;
  if (U > 0.0) {
    double sum = 0.0;
    for (int k = threadIdx.x; k < g.K; k += kThreads) sum += pow((cone(g, s, k, x, y) + dphi) / U, g.p);
    sum = block_sum(sum);
    norm = U * pow(sum, 1.0 / g.p);
  }
  if (want_a) {
    double a = 0.0;
    if (norm > 0.0)
      for (int k = threadIdx.x; k < g.K; k += kThreads) a += pow((cone(g, s, k, x, y) + dphi) / norm, g.p - 1.0);
    a = block_sum(a);
    if (threadIdx.x == 0) w.A[j] = a;
  }
  if (threadIdx.x == 0) {
    w.F[j] = norm - dphi;
    w.norm[j] = norm;
  }
}

// 4. M = max |F| and its node (single block)
__global__ void fmax_kernel(Geo g, Work w) {
  double bv = -1.0;
  long long bi = LLONG_MAX;
  for (int j = threadIdx.x; j < g.J; j += kThreads)
    if (better_max(fabs(w.F[j]), j, bv, bi)) { bv = fabs(w.F[j]); bi = j; }
  block_argext<true>(bv, bi);
  if (threadIdx.x == 0) {
    w.sc[S_BIGM] = bv;
    w.sc[S_JM] = (double)bi;
  }
}

template <typename T>
__global__ void write_phi_kernel(Geo g, Work w, T* phi) {
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j >= g.J) return;
  double x, y;
  long long n;
  node_of(g, j, x, y, n);
  phi[n] = (T)(w.F[j] / w.sc[S_BIGM]);
}

// 5. H_j = dJ/dF_j: sum_i g_i F_i first (single block), then H
template <typename T>
__global__ void gf_kernel(Geo g, Work w, const T* dJdphi) {
  double acc = 0.0;
  for (int j = threadIdx.x; j < g.J; j += kThreads) {
    double x, y;
    long long n;
    node_of(g, j, x, y, n);
    acc += (double)dJdphi[n] * w.F[j];
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) w.sc[S_GF] = acc;
}

template <typename T>
__global__ void h_kernel(Geo g, Work w, const T* dJdphi) {
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j >= g.J) return;
  double x, y;
  long long n;
  node_of(g, j, x, y, n);
  const double M = w.sc[S_BIGM];
  double h = (double)dJdphi[n] / M;
  if (j == (int)w.sc[S_JM]) h += (w.F[j] > 0 ? 1.0 : (w.F[j] < 0 ? -1.0 : 0.0)) * (-w.sc[S_GF] / (M * M));
  w.H[j] = h;
}

// 6. dJ/d(dphi) = sum_j H_j (A_j - 1) (single block)
__global__ void ddphi_kernel(Geo g, Work w) {
  double acc = 0.0;
  for (int j = threadIdx.x; j < g.J; j += kThreads) acc += w.H[j] * (w.A[j] - 1.0);
  acc = block_sum(acc);
  if (threadIdx.x == 0) w.sc[S_DDPHI] = acc;
}

// 7. dJ/ds_k = sum_j H_j W_jk (+ the shift term at the minimising RBF)
__global__ void ds_kernel(Geo g, const double* s, Work w, double* dJds) {
  const int k = blockIdx.x;
  const double dphi = w.sc[S_DPHI];
  double acc = 0.0;
  for (int j = threadIdx.x; j < g.J; j += kThreads) {
    const double nj = w.norm[j];
    if (!(nj > 0.0)) continue;
    double x, y;
    long long n;
    node_of(g, j, x, y, n);
    acc += w.H[j] * pow((cone(g, s, k, x, y) + dphi) / nj, g.p - 1.0);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    const double m = w.sc[S_M];
    if (k == (int)w.sc[S_KM]) acc += w.sc[S_DDPHI] * (m > 0 ? 1.0 : (m < 0 ? -1.0 : 0.0));
    dJds[k] = acc;
  }
}

__global__ void adam_kernel(double* s, const double* gr, double* m, double* v, int n, double lr, double b1,
                            double b2, double eps, double c1, double c2) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const double g = gr[i];
  const double mi = b1 * m[i] + (1.0 - b1) * g;
  const double vi = b2 * v[i] + (1.0 - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  s[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
}

bool make_geo(const llg_rbf* r, Geo& g) {
  if (!r || r->nx < 1 || r->ny < 1 || !(r->dx > 0) || !(r->dy > 0) || r->nrx < 1 || r->nry < 1 || !(r->p >= 1.0))
    return false;
  const int* b = r->box;
  if (b[0] < 0 || b[1] > r->nx || b[0] >= b[1] || b[2] < 0 || b[3] > r->ny || b[2] >= b[3]) return false;
  g.nx = r->nx;
  for (int i = 0; i < 4; ++i) g.box[i] = b[i];
  g.nrx = r->nrx;
  g.nry = r->nry;
  g.J = (b[1] - b[0]) * (b[3] - b[2]);
  g.K = r->nrx * r->nry;
  g.dx = r->dx;
  g.dy = r->dy;
  g.hx = ((double)(b[1] - b[0]) * r->dx) / (double)r->nrx;
  g.hy = ((double)(b[3] - b[2]) * r->dy) / (double)r->nry;
  g.c = g.hx < g.hy ? g.hx : g.hy;
  g.p = r->p;
  return true;
}

llg_status map_kernels(const Geo& g, const double* s, Work w, bool want_a, cudaStream_t st) {
  kmin_kernel<<<g.K, kThreads, 0, st>>>(g, s, w);
  shift_kernel<<<1, kThreads, 0, st>>>(g, w);
  norm_kernel<<<g.J, kThreads, 0, st>>>(g, s, w, want_a ? 1 : 0);
  fmax_kernel<<<1, kThreads, 0, st>>>(g, w);
  return cudaGetLastError() == cudaSuccess ? LLG_OK : LLG_ECUDA;
}

}  // namespace

extern "C" {

size_t llg_rbf_workspace_bytes(const llg_rbf* r) {
  Geo g;
  if (!make_geo(r, g)) return 0;
  return sizeof(double) * ((size_t)4 * g.J + 2 * (size_t)g.K + S_COUNT);
}

llg_status llg_rbf_phi(const llg_rbf* r, const double* s_dev, void* phi_dev, int precision, void* work_dev,
                       void* cuda_stream) {
  Geo g;
  if (!make_geo(r, g) || !s_dev || !phi_dev || !work_dev || (precision != LLG_FP32 && precision != LLG_FP64))
    return LLG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  Work w = carve(work_dev, g.J, g.K);
  if (llg_status e = map_kernels(g, s_dev, w, false, st)) return e;
  const int nb = (g.J + kThreads - 1) / kThreads;
  if (precision == LLG_FP32)
    write_phi_kernel<float><<<nb, kThreads, 0, st>>>(g, w, static_cast<float*>(phi_dev));
  else
    write_phi_kernel<double><<<nb, kThreads, 0, st>>>(g, w, static_cast<double*>(phi_dev));
  return cudaGetLastError() == cudaSuccess ? LLG_OK : LLG_ECUDA;
}

llg_status llg_rbf_grad(const llg_rbf* r, const double* s_dev, const void* dJdphi_dev, int precision,
                        double* dJds_dev, void* work_dev, void* cuda_stream) {
  Geo g;
  if (!make_geo(r, g) || !s_dev || !dJdphi_dev || !dJds_dev || !work_dev ||
      (precision != LLG_FP32 && precision != LLG_FP64))
    return LLG_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  Work w = carve(work_dev, g.J, g.K);
  if (llg_status e = map_kernels(g, s_dev, w, true, st)) return e;
  const int nb = (g.J + kThreads - 1) / kThreads;
  if (precision == LLG_FP32) {
    const float* d = static_cast<const float*>(dJdphi_dev);
    gf_kernel<float><<<1, kThreads, 0, st>>>(g, w, d);
    h_kernel<float><<<nb, kThreads, 0, st>>>(g, w, d);
  } else {
    const double* d = static_cast<const double*>(dJdphi_dev);
    gf_kernel<double><<<1, kThreads, 0, st>>>(g, w, d);
    h_kernel<double><<<nb, kThreads, 0, st>>>(g, w, d);
  }
  ddphi_kernel<<<1, kThreads, 0, st>>>(g, w);
  ds_kernel<<<g.K, kThreads, 0, st>>>(g, s_dev, w, dJds_dev);
  return cudaGetLastError() == cudaSuccess ? LLG_OK : LLG_ECUDA;
}

llg_status llg_adam_step(double* s_dev, const double* grad_dev, double* m_dev, double* v_dev, int n, long long t,
                         double lr, double b1, double b2, double eps, void* cuda_stream) {
  if (!s_dev || !grad_dev || !m_dev || !v_dev || n < 1 || t < 1 || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1))
    return LLG_EINVAL;
  const double c1 = 1.0 - std::pow(b1, (double)t), c2 = 1.0 - std::pow(b2, (double)t);
  adam_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      s_dev, grad_dev, m_dev, v_dev, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? LLG_OK : LLG_ECUDA;
}

}  // extern "C"
