// Demagnetising-tensor setup, FP64 on the device (once per grid shape).
//
// N(r) is the cell-averaged demagnetising tensor of two dx*dy*dz cuboids at
// offset r (the demag term of the effective field, Methods).  Near the
// origin it is Newell, Williams and Dunlop's closed form, a 27-point second
// difference of their functions f and g; that form cancels ~(|r|/h)^6 digits,
// so from |r| >= 6 max(dx,dy,dz) on the tensor is integrated instead: the
// dipole kernel (I - 3 u u^T)/(4 pi |u|^3) against the tent-shaped overlap
// density of the two cells, 6 Gauss-Legendre points per half tent per axis.
//
// The tensor is written, with its parity signs, onto the zero-padded
// Px x Py grid at offsets modulo (Px, Py); complex FFTs of the rows and then
// the columns give its spectrum, which is real (each component is even or
// odd in every coordinate).  The packed table holds, for kx in [0, Px/2] and
// ky in [0, Py/2], the four 2D components (xx, yy, zz, xy) scaled by
// -mu0/(Px Py), so that one forward FFT of M = Ms psi m, the product and an
// unnormalised inverse FFT give B_d directly.
#include "common.cuh"
#include "fft.cuh"

namespace llg {

__device__ __forceinline__ double asinh_ratio(double num, double den) {
  return den > 0.0 ? asinh(num / den) : 0.0;
}
__device__ __forceinline__ double atan_ratio(double num, double den) {
  return den > 0.0 ? atan(num / den) : 0.0;
}

// Newell f: even in every argument.
__device__ double newell_f(double x, double y, double z) {
  x = fabs(x); y = fabs(y); z = fabs(z);
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = sqrt(x2 + y2 + z2);
  double t = 0.5 * y * (z2 - x2) * asinh_ratio(y, sqrt(x2 + z2));
  t += 0.5 * z * (y2 - x2) * asinh_ratio(z, sqrt(x2 + y2));
  t -= x * y * z * atan_ratio(y * z, x * R);
  t += (2.0 * x2 - y2 - z2) * R / 6.0;
  return t;
}

// Newell g: odd in x and y, even in z.
__device__ double newell_g(double x, double y, double z) {
  const double sgn = (x < 0 ? -1.0 : (x > 0 ? 1.0 : 0.0)) * (y < 0 ? -1.0 : (y > 0 ? 1.0 : 0.0));
  x = fabs(x); y = fabs(y); z = fabs(z);
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = sqrt(x2 + y2 + z2);
  double t = x * y * z * asinh_ratio(z, sqrt(x2 + y2));
  t += y / 6.0 * (3.0 * z2 - y2) * asinh_ratio(x, sqrt(y2 + z2));
  t += x / 6.0 * (3.0 * z2 - x2) * asinh_ratio(y, sqrt(x2 + z2));
  t -= z2 * z / 6.0 * atan_ratio(x * y, z * R);
  t -= z * y2 / 2.0 * atan_ratio(x * z, y * R);
  t -= z * x2 / 2.0 * atan_ratio(y * z, x * R);
  t -= x * y * R / 3.0;
  return sgn * t;
}

template <bool OFFDIAG>
__device__ double second_difference(double X, double Y, double Z, double dx, double dy, double dz) {
  const double w[3] = {-1.0, 2.0, -1.0};
  double s = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        const double a = X + (i - 1) * dx, b = Y + (j - 1) * dy, c = Z + (k - 1) * dz;
        s += w[i] * w[j] * w[k] * (OFFDIAG ? newell_g(a, b, c) : newell_f(a, b, c));
      }
  return s / (4.0 * M_PI * dx * dy * dz);
}

// 6-point Gauss-Legendre rule on [-1, 1] (nodes, weights).
__constant__ double kGLx[6] = {-0.9324695142031521, -0.6612093864662645, -0.2386191860831969,
                               0.2386191860831969, 0.6612093864662645, 0.9324695142031521};
__constant__ double kGLw[6] = {0.1713244923791704, 0.3607615730481386, 0.4679139345726910,
                               0.4679139345726910, 0.3607615730481386, 0.1713244923791704};

// Node s and weight of point q (0..11) of the tent rule on [-h, h] with
// density (h - |s|)/h^2: 6 points on each half.
__device__ __forceinline__ void tent_point(int q, double h, double* s, double* wt) {
  const int k = q % 6;
  const double t = kGLx[k];
  const double u = 0.5 * h * (t + 1.0);            // in [0, h]
  const double w = (h - u) / (h * h) * 0.5 * h * kGLw[k];
  *s = (q < 6) ? -u : u;
  *wt = w;
}

// Components (xx, yy, zz, xy, xz, yz) at integer offsets.
__device__ void tensor_at(int ix, int iy, int iz, double dx, double dy, double dz, double out[6]) {
  const double X = ix * dx, Y = iy * dy, Z = iz * dz;
  const double hmax = fmax(dx, fmax(dy, dz));
  const double r2 = X * X + Y * Y + Z * Z;
  if (r2 < 36.0 * hmax * hmax) {
    out[0] = second_difference<false>(X, Y, Z, dx, dy, dz);
    out[1] = second_difference<false>(Y, X, Z, dy, dx, dz);
    out[2] = second_difference<false>(Z, Y, X, dz, dy, dx);
    out[3] = second_difference<true>(X, Y, Z, dx, dy, dz);
    out[4] = second_difference<true>(X, Z, Y, dx, dz, dy);
    out[5] = second_difference<true>(Y, Z, X, dy, dz, dx);
    return;
  }
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int a = 0; a < 12; ++a) {
    double sa, wa;
    tent_point(a, dx, &sa, &wa);
    for (int b = 0; b < 12; ++b) {
      double sb, wb;
      tent_point(b, dy, &sb, &wb);
      for (int c = 0; c < 12; ++c) {
        double sc, wc;
        tent_point(c, dz, &sc, &wc);
        const double u = X + sa, v = Y + sb, w = Z + sc;
        const double q2 = u * u + v * v + w * w;
        const double k = wa * wb * wc / (4.0 * M_PI * q2 * sqrt(q2));
        const double iq = 3.0 / q2;
        acc[0] += k * (1.0 - iq * u * u);
        acc[1] += k * (1.0 - iq * v * v);
        acc[2] += k * (1.0 - iq * w * w);
        acc[3] -= k * iq * u * v;
        acc[4] -= k * iq * u * w;
        acc[5] -= k * iq * v * w;
      }
    }
  }
  const double V = dx * dy * dz;
  for (int i = 0; i < 6; ++i) out[i] = V * acc[i];
}

// Real-space tensor on the padded grid G[NC][Pz][Py][Px] (complex, imag = 0),
// from the octant ix in [0,nx), iy in [0,ny), iz in [0,nz), mirrored to the
// negative offsets with each component's parity.  NC = 4 (film: xx, yy, zz,
// xy, one layer) or 6 (3D: xx, yy, zz, xy, xz, yz).
__global__ void tensor_fill_kernel(double2* G, int NC, int nx, int ny, int nz, int Px, int Py, int Pz, double dx,
                                   double dy, double dz) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nx * ny * nz) return;
  const int ix = (int)(idx % nx), iy = (int)((idx / nx) % ny), iz = (int)(idx / ((long long)nx * ny));
  double t[6];
  tensor_at(ix, iy, iz, dx, dy, dz, t);
  const long long plane = (long long)Px * Py, vol = plane * Pz;
  for (int sx = 0; sx < 2; ++sx) {
    if (sx == 1 && ix == 0) continue;
    for (int sy = 0; sy < 2; ++sy) {
      if (sy == 1 && iy == 0) continue;
      for (int sz = 0; sz < 2; ++sz) {
        if (sz == 1 && iz == 0) continue;
        const int px = sx ? Px - ix : ix;
        const int py = sy ? Py - iy : iy;
        const int pz = sz ? Pz - iz : iz;
        // xy odd in x and y, xz odd in x and z, yz odd in y and z
        const double sgn[6] = {1.0, 1.0, 1.0, (sx ^ sy) ? -1.0 : 1.0, (sx ^ sz) ? -1.0 : 1.0,
                               (sy ^ sz) ? -1.0 : 1.0};
        const long long o = (long long)pz * plane + (long long)py * Px + px;
        for (int c = 0; c < NC; ++c) G[c * vol + o] = make_double2(sgn[c] * t[c], 0.0);
      }
    }
  }
}

// In-place complex FFTs of `nlines` lines of length L = 2^log2L; element e of
// line l sits at data[l_base(l) + e * estride] with l_base = (l / inner) *
// outer_stride + (l % inner) * inner_stride.
__global__ void fft_lines_kernel(double2* data, int log2L, int nlines, long long estride, int inner,
                                 long long inner_stride, long long outer_stride,
                                 const double2* __restrict__ tw) {
  extern __shared__ double2 sbuf[];
  const int L = 1 << log2L;
  const int l = blockIdx.x;
  if (l >= nlines) return;
  const long long base = (long long)(l / inner) * outer_stride + (long long)(l % inner) * inner_stride;
  double2* a = sbuf;
  double2* b = sbuf + L;
  for (int e = threadIdx.x; e < L; e += blockDim.x) a[e] = data[base + e * estride];
  __syncthreads();
  double2* r = fft_batch<double2, -1>(a, b, log2L, 1, tw);
  for (int e = threadIdx.x; e < L; e += blockDim.x) data[base + e * estride] = r[e];
}

// Packed table [kx 0..Px/2][ky 0..Py/2][4] of -mu0/(Px Py) * Re(G^).  The xy
// component is odd in both coordinates, so it vanishes exactly on the kx = 0,
// kx = Px/2, ky = 0 and ky = Py/2 lines; those entries are set to zero.
// Record (kx, ky) lives at table[(kx nky + ky) 4 + c]; a double-float
// table stores each column kx planar, its nky hi records (4 floats each)
// then its nky lo records, in the same 8 floats per record of space.
template <typename T>
__device__ __forceinline__ void tensor_put(T* table, int kx, int ky, int nky, int c, double v) {
  table[((long long)kx * nky + ky) * 4 + c] = (T)v;
}
template <>
__device__ __forceinline__ void tensor_put<dfloat>(dfloat* table, int kx, int ky, int nky, int c, double v) {
  const dfloat d(v);
  float* col = reinterpret_cast<float*>(table) + (long long)kx * nky * 8;
  col[ky * 4 + c] = d.hi;
  col[(nky + ky) * 4 + c] = d.lo;
}

template <typename T>
__global__ void tensor_pack_kernel(const double2* G, T* table, int Px, int Py) {
  const int nkx = Px / 2 + 1, nky = Py / 2 + 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nkx * nky) return;
  const int kx = idx / nky, ky = idx % nky;
  const long long plane = (long long)Px * Py;
  const double scale = -kMu0 / ((double)Px * (double)Py);
  for (int c = 0; c < 4; ++c) {
    double v = G[c * plane + (long long)ky * Px + kx].x * scale;
    if (c == 3 && (kx == 0 || kx == Px / 2 || ky == 0 || ky == Py / 2)) v = 0.0;
    tensor_put(table, kx, ky, nky, c, v);
  }
}

// 3D table [kz 0..Pz/2][kx 0..Px/2][ky 0..Py/2][8]: xx, yy, zz, xy, xz, yz
// of -mu0/(Px Py Pz) * Re(G^), then two zeros (32/64-byte records).  An odd
// component vanishes exactly where the sine of one of its odd coordinates
// does (index 0 or the Nyquist index); those entries are set to zero.
template <typename T>
__global__ void tensor_pack3_kernel(const double2* G, T* table, int Px, int Py, int Pz) {
  const int nkx = Px / 2 + 1, nky = Py / 2 + 1, nkz = Pz / 2 + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nkx * nky * nkz) return;
  const int ky = (int)(idx % nky), kx = (int)((idx / nky) % nkx), kz = (int)(idx / ((long long)nky * nkx));
  const long long plane = (long long)Px * Py, vol = plane * Pz;
  const double scale = -kMu0 / ((double)Px * (double)Py * (double)Pz);
  const bool ex = kx == 0 || kx == Px / 2, ey = ky == 0 || ky == Py / 2, ez = kz == 0 || kz == Pz / 2;
  const bool zero[6] = {false, false, false, ex || ey, ex || ez, ey || ez};
  const long long o = (long long)kz * plane + (long long)ky * Px + kx;
  for (int c = 0; c < 6; ++c) table[idx * 8 + c] = zero[c] ? (T)0 : (T)(G[c * vol + o].x * scale);
  table[idx * 8 + 6] = (T)0;
  table[idx * 8 + 7] = (T)0;
}

template __global__ void tensor_pack_kernel<float>(const double2*, float*, int, int);
template __global__ void tensor_pack_kernel<double>(const double2*, double*, int, int);
template __global__ void tensor_pack3_kernel<float>(const double2*, float*, int, int, int);
template __global__ void tensor_pack3_kernel<double>(const double2*, double*, int, int, int);
template __global__ void tensor_pack_kernel<dfloat>(const double2*, dfloat*, int, int);
template __global__ void tensor_pack3_kernel<dfloat>(const double2*, dfloat*, int, int, int);

// Elements of T in the packed spectrum table of one grid shape.
long long tensor_table_len(int Px, int Py, int Pz) {
  if (Pz <= 1) return (long long)(Px / 2 + 1) * (Py / 2 + 1) * 4;
  return (long long)(Px / 2 + 1) * (Py / 2 + 1) * (Pz / 2 + 1) * 8;
}

// Complex FP64 scratch the build of one grid shape needs.
long long tensor_scratch_len(int Px, int Py, int Pz) {
  return (long long)(Pz <= 1 ? 4 : 6) * Px * Py * (Pz <= 1 ? 1 : Pz);
}

// Host entry: build the packed spectrum of one grid shape into `table`
// (device, tensor_table_len(Px, Py, Pz) elements of T; Pz = 1 for a film).
// G is FP64 scratch of tensor_scratch_len(Px, Py, Pz) complex values; tw the
// FP64 twiddle table.
template <typename T>
cudaError_t build_tensor_spectrum(T* table, double2* G, int nx, int ny, int nz, int Px, int Py, int Pz,
                                  double dx, double dy, double dz, const double2* tw, cudaStream_t st) {
  const int NC = Pz <= 1 ? 4 : 6;
  if (Pz < 1) Pz = 1;
  const long long plane = (long long)Px * Py, vol = plane * Pz;
  cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double2) * NC * vol, st);
  if (e != cudaSuccess) return e;
  const long long n = (long long)nx * ny * nz;
  tensor_fill_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(G, NC, nx, ny, nz, Px, Py, Pz, dx, dy, dz);
  int lx = 0, ly = 0, lz = 0;
  while ((1 << lx) < Px) ++lx;
  while ((1 << ly) < Py) ++ly;
  while ((1 << lz) < Pz) ++lz;
  const size_t shx = 2 * sizeof(double2) * Px, shy = 2 * sizeof(double2) * Py;
  cudaFuncSetAttribute(fft_lines_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(shx > shy ? shx : shy));
  // x lines: NC Pz Py contiguous lines
  const int nlx = (int)(NC * Pz * Py);
  fft_lines_kernel<<<nlx, 256, shx, st>>>(G, lx, nlx, 1, nlx, Px, 0, tw);
  // y lines, stride Px: line l -> plane l / Px (component and layer), column l % Px
  const int nly = (int)(NC * Pz * Px);
  fft_lines_kernel<<<nly, 256, shy, st>>>(G, ly, nly, Px, Px, 1, plane, tw);
  if (Pz > 1) {
    // z lines, stride Px Py: line l -> component l / plane, point l % plane
    const int nlz = (int)(NC * plane);
    fft_lines_kernel<<<nlz, 64, 2 * sizeof(double2) * Pz, st>>>(G, lz, nlz, plane, (int)plane, 1, vol, tw);
    const long long nk = (long long)(Px / 2 + 1) * (Py / 2 + 1) * (Pz / 2 + 1);
    tensor_pack3_kernel<T><<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(G, table, Px, Py, Pz);
  } else {
    const int nk = (Px / 2 + 1) * (Py / 2 + 1);
    tensor_pack_kernel<T><<<(nk + 255) / 256, 256, 0, st>>>(G, table, Px, Py);
  }
  return cudaGetLastError();
}

template cudaError_t build_tensor_spectrum<float>(float*, double2*, int, int, int, int, int, int, double, double,
                                                  double, const double2*, cudaStream_t);
template cudaError_t build_tensor_spectrum<double>(double*, double2*, int, int, int, int, int, int, double, double,
                                                   double, const double2*, cudaStream_t);
template cudaError_t build_tensor_spectrum<dfloat>(dfloat*, double2*, int, int, int, int, int, int, double, double,
                                                   double, const double2*, cudaStream_t);

}  // namespace llg
