// Common device types of the LLG solver: complex arithmetic, the per-instance
// descriptor and the work-tile tables shared by every kernel.
#pragma once
#include <cmath>

#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"

namespace llg {

constexpr double kMu0 = 1.2566370614359173e-06;     // 4 pi 1e-7
constexpr double kGamma = 1.76085963023e11;         // rad s^-1 T^-1
constexpr int kTwiddleN = 4096;                      // W_4096^k table length
constexpr int kMaxLx = 1024;                         // complex row FFT length (nx <= 1024)
constexpr int kMaxPy = 1024;                         // column FFT length
constexpr int kMaxNz = 8;                            // layers of a 3D grid (padded z length <= 16)

// Shared-memory index of element i of an FFT sequence: one pad slot per
// eight elements spreads strided accesses over the banks.
__host__ __device__ constexpr int rf_pad(int i) { return i + (i >> 3); }
__host__ __device__ constexpr int rf_padded_len(int L) { return L + (L >> 3); }
// Padding of the row-family sequences and of every register FFT's internal
// exchanges: one slot per 16 once a sequence's L/8 lanes fill whole
// half-warps (L >= 128), so that natural-order accesses by 16 consecutive
// lanes (8-byte elements, 16 bank pairs per wavefront) and the radix-2/4
// pass writes meet no bank twice; one per 8 below that.
__host__ __device__ constexpr int row_pad(int L, int i) { return L >= 128 ? i + (i >> 4) : i + (i >> 3); }
__host__ __device__ constexpr int row_padded_len(int L) { return L >= 128 ? L + (L >> 4) : L + (L >> 3); }

// Padded z length of the demag convolution: 1 for a film, else the power of
// two >= 2 nz (any length >= 2 nz - 1 gives the same linear convolution).
__host__ __device__ constexpr int pz_of(int nz) {
  return nz <= 1 ? 1 : (nz <= 2 ? 4 : (nz <= 4 ? 8 : 16));
}

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<dfloat> { using type = dcplx; };
template <typename T> using cplx = typename Cplx<T>::type;

// Shared-memory layout of a register-FFT sequence by element type.  FP32 and
// FP64 take row_pad.  The 16-byte double-float elements take one pad slot per
// 8 at every length: a quarter-warp's 8 lanes then fill the 32 banks once,
// for the stride-2/4/8 writes of every pass as for natural order.
template <typename C> struct SeqPad {
  __host__ __device__ static constexpr int pad(int L, int i) { return row_pad(L, i); }
  __host__ __device__ static constexpr int len(int L) { return row_padded_len(L); }
};
template <> struct SeqPad<dcplx> {
  __host__ __device__ static constexpr int pad(int, int i) { return i + (i >> 3); }
  __host__ __device__ static constexpr int len(int L) { return L + (L >> 3); }
};
template <typename C> __host__ __device__ constexpr int seq_pad(int L, int i) { return SeqPad<C>::pad(L, i); }
// Row-family group stride: the padded length rounded up to even (every
// sequence starts on a 16-byte boundary).
template <typename C> __host__ __device__ constexpr int seq_group_stride(int L) { return (SeqPad<C>::len(L) + 1) & ~1; }
// Entries of the per-pass twiddle table that the double-float (rolled)
// transforms of length L read after their W table: fewer than L.
template <typename S> __host__ __device__ constexpr int pass_tw_len(int) { return 0; }
template <> __host__ __device__ constexpr int pass_tw_len<dfloat>(int L) { return L; }

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C> __host__ __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename C> __host__ __device__ __forceinline__ C mul_mi(C a) { return mk<C>(a.y, -a.x); }
template <typename C> __host__ __device__ __forceinline__ C mul_pi(C a) { return mk<C>(-a.y, a.x); }

// FP32 complex sums and real scalings as packed FP32x2 operations (one
// instruction for both parts on sm_100 and later; the same round-to-nearest
// result per part as two scalar operations).  Declared before the FFT
// templates so that their calls on float2 resolve here.
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fmul2_rn(a, make_float2(s, s));
#else
  return make_float2(a.x * s, a.y * s);
#endif
}

// Block-wide sum of a double; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
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

// Per-instance coefficients in the compute precision T, converted on the host
// so that no kernel converts a double inside its node loop (the FP64 pipe of
// this GPU is narrow; a conversion per node and term showed up as a third
// of the issue slots of the FP32 stage kernel).
template <typename T>
struct Coef {
  T Ms, cx, cy, cz, kan;
  T ku[3], B_bias[3], rf_dir[3];
  T alpha, alpha_edge;   // Gilbert damping inside and at the absorbing edge
  T absorb_w, inv_absorb_w;  // ramp width in nodes and its reciprocal
  T gp0;                 // -gamma/(1+alpha^2) for the interior damping
  T wbox[2];
  T A, V, escale, ihx2, ihy2, ihz2;
};

// Per-instance descriptor (device copy).  Offsets are in elements of the
// pooled arrays; every node offset is a multiple of 4.
struct DevInst {
  int nx, ny, nz;
  int Lx, Py;            // complex row FFT length (Px/2) and column FFT length
  int log2Lx, log2Py;
  int Pz;                // padded z length: 1 for a film (nz = 1), else 2^k >= 2 nz
  int shape;             // index of the demag spectrum table
  int ntile, tile_off;   // row tiles of this instance, index of its first row tile
  long long nodes;       // nx*ny*nz
  long long layer;       // nx*ny: node stride between z layers
  long long node_off;    // offset into node arrays (per component block: 3*nodes)
  long long spec_off;    // offset into the spectrum pool, complex elements
  long long tens_off;    // offset into the tensor pool, real elements
  long long slot_off;    // offset into the objective partials: (nsteps+1) x ntile
  long long rf_off;      // offset into the RF drive table (3 nsteps + 3 values)
  long long wt_off;      // spectral / curve objective: offset into the per-step weights ((nsteps+1) x 2)
  double Ms;
  double cex_x, cex_y, cex_z;   // 2A/(Ms h^2)
  double kan;                   // 2Ku/Ms
  double ku[3];
  double alpha, alpha_edge;
  int absorb_nodes, absorb_x, absorb_y;
  int src[4];
  double B_bias[3];
  double b_rf, f_rf;
  double rf_dir[3];
  double sigmoid_a;
  int objective, comp, power;
  int boxes[2][4];
  double wbox[2];               // w_b / |box b|
  double V;                     // cell volume
  double ihx2, ihy2, ihz2;      // 1/dx^2, 1/dy^2, 1/dz^2
  double escale;                // 1/(K_d V_domain)
  double A;                     // exchange constant
  double area_target, penalty_w;
  double centre_w, centre_x0, centre_y0;   // curve objective: centre term (node-index units)
  Coef<double> cd;              // the coefficients above in FP64 ...
  Coef<float> cf;               // ... and rounded to FP32
};

template <typename T> __device__ __forceinline__ const Coef<T>& coef(const DevInst& I);
template <> __device__ __forceinline__ const Coef<double>& coef<double>(const DevInst& I) { return I.cd; }
template <> __device__ __forceinline__ const Coef<float>& coef<float>(const DevInst& I) { return I.cf; }

// Fill both coefficient sets from the FP64 fields of a descriptor.  gp0 is
// formed with one fused multiply-add, as the device forms -gamma/(1+a^2).
template <typename T>
inline void fill_coef_t(Coef<T>& k, const DevInst& d) {
  k.Ms = (T)d.Ms; k.cx = (T)d.cex_x; k.cy = (T)d.cex_y; k.cz = (T)d.cex_z; k.kan = (T)d.kan;
  for (int c = 0; c < 3; ++c) {
    k.ku[c] = (T)d.ku[c];
    k.B_bias[c] = (T)d.B_bias[c];
    k.rf_dir[c] = (T)d.rf_dir[c];
  }
  k.alpha = (T)d.alpha;
  k.alpha_edge = (T)d.alpha_edge;
  k.absorb_w = (T)d.absorb_nodes;
  k.inv_absorb_w = d.absorb_nodes > 0 ? (T)1 / k.absorb_w : (T)0;
  k.gp0 = -(T)kGamma / std::fma(k.alpha, k.alpha, (T)1);
  k.wbox[0] = (T)d.wbox[0];
  k.wbox[1] = (T)d.wbox[1];
  k.A = (T)d.A; k.V = (T)d.V; k.escale = (T)d.escale;
  k.ihx2 = (T)d.ihx2; k.ihy2 = (T)d.ihy2; k.ihz2 = (T)d.ihz2;
}
inline void fill_coef(DevInst& d) {
  fill_coef_t(d.cd, d);
  fill_coef_t(d.cf, d);
}

// Cooperative copy of a descriptor into shared memory (all threads call it).
__device__ __forceinline__ void load_inst(DevInst& dst, const DevInst* src) {
  static_assert(sizeof(DevInst) % 4 == 0, "descriptor must be word sized");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(DevInst) / 4); i += blockDim.x) d[i] = s[i];
}

// Rows per row tile for a row FFT of length L: 3 x L/8 threads per row in a
// 384-thread block (every thread then owns a row slot).
__host__ __device__ constexpr int rows_per_tile(int L) { return 1024 / L; }

// FFT exchange scratch of every stage kernel, complex values: the row kernels
// use R = 1024/L row slots x 3 components x (padded length rounded to even),
// the column kernel 3 x 1024/L groups of (padded length + 1); both <= 3840.
constexpr int kExch = 3840;

// Dynamic shared memory of the stage and adjoint kernels for a row FFT of
// length L on rows of nx nodes: exchange scratch, the staged halo rows (4
// resp. 7 node arrays over R+2 rows) and the W_{2L} table.
template <typename T>
__host__ __device__ constexpr size_t stage_smem_bytes(int L, int nx) {
  return (size_t)kExch * sizeof(cplx<T>) + (size_t)4 * (rows_per_tile(L) + 2) * nx * sizeof(T) +
         (size_t)2 * L * sizeof(cplx<T>);
}
// S: the real type of the adjoint's frequency domain (T, or dfloat).
template <typename T, typename S = T>
__host__ __device__ constexpr size_t adj_smem_bytes(int L, int nx) {
  return (size_t)kExch * sizeof(cplx<S>) + (size_t)7 * (rows_per_tile(L) + 2) * nx * sizeof(T) +
         (size_t)(2 * L + pass_tw_len<S>(L)) * sizeof(cplx<S>);
}


// Row tile: rows y0 .. y0+nrows-1 of layer z of instance `inst` (a tile never
// spans two layers); k is the tile's index within its instance (the slot of
// its partial sums, which are added in tile order afterwards so that J does
// not depend on the order tiles finish).
struct RowTile { int inst, z, y0, nrows, k; };

// First node of a row tile in the instance-pooled node arrays.
__host__ __device__ __forceinline__ long long tile_base(const DevInst& I, const RowTile& t) {
  return I.node_off + ((long long)t.z * I.ny + t.y0) * I.nx;
}
// Column tile: complex columns kx0 .. kx0+ncols-1 of instance `inst`.
struct ColTile { int inst, kx0, ncols, pad; };

}  // namespace llg
