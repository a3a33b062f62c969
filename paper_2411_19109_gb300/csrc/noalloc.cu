// llg_field_noalloc: the effective-field evaluation of llg_field for one
// FP32 instance, with every scratch buffer in a fixed device array of this
// file instead of memory obtained from the CUDA allocator.
//
// Who needs it: code that must not allocate device memory at the point
// where it wants a field evaluation -- a host application or framework that
// owns all device memory through its own allocator and budget, or a
// latency-critical loop where the implicit synchronisation of
// cudaMalloc/cudaFree would stall other streams.  The caller still provides
// phi, m and the output B.
//
// The scratch below (about 5.3 MB) is a static __device__ object: every GPU
// that loads this library holds it until the process exits.  It bounds the
// grid to NA_MAX_N x NA_MAX_N nodes.  In host code the array's name is only a
// host-side stand-in; its device address is looked up with
// cudaGetSymbolAddress on every call (a host-side lookup) and carved into the
// buffers the kernels use.  The twiddle tables are uploaded once per device,
// and again if the address changes (a new context after a device reset).
// Each call's descriptor and work tiles reach the device as kernel
// arguments of a set-up kernel, not as copies from host memory.  The demag
// spectrum is rebuilt only when the grid or cell size differs from the
// previous call's on that device.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "kernels.cuh"
#include "llg.h"

using namespace llg;

namespace {

constexpr int NA_MAX_N = 128;                  // max nx and ny
constexpr int NA_PX = 2 * NA_MAX_N;            // padded extents at the maximum
constexpr int NA_PY = 2 * NA_MAX_N;
constexpr int NA_LX = NA_PX / 2;
constexpr int NA_MAX_ROW_TILES = NA_MAX_N;     // at most one row tile per row
constexpr int NA_MAX_COL_TILES = NA_LX;        // at most one column tile per column

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// region sizes in bytes
constexpr size_t SZ_G = align256(sizeof(double2) * 4 * NA_PX * NA_PY);                     // FP64 tensor grid
constexpr size_t SZ_TENS = align256(sizeof(float) * 4 * (NA_PX / 2 + 1) * (NA_PY / 2 + 1));  // tensor spectrum
constexpr size_t SZ_SPEC = align256(sizeof(float2) * 3 * NA_MAX_N * NA_LX);                  // row spectra
constexpr size_t SZ_PSI = align256(sizeof(float) * NA_MAX_N * NA_MAX_N);                     // psi, dpsi
constexpr size_t SZ_TW = align256(sizeof(float2) * kTwiddleN);
constexpr size_t SZ_TW64 = align256(sizeof(double2) * kTwiddleN);
constexpr size_t SZ_INST = align256(sizeof(DevInst));
constexpr size_t SZ_RT = align256(sizeof(RowTile) * NA_MAX_ROW_TILES);
constexpr size_t SZ_CT = align256(sizeof(ColTile) * NA_MAX_COL_TILES);
constexpr size_t SZ_SUM = align256(sizeof(double) * NA_MAX_ROW_TILES);                        // psi partials

constexpr size_t OFF_G = 0;
constexpr size_t OFF_TENS = OFF_G + SZ_G;
constexpr size_t OFF_SPEC = OFF_TENS + SZ_TENS;
constexpr size_t OFF_PSI = OFF_SPEC + SZ_SPEC;
constexpr size_t OFF_DPSI = OFF_PSI + SZ_PSI;
constexpr size_t OFF_TW = OFF_DPSI + SZ_PSI;
constexpr size_t OFF_TW64 = OFF_TW + SZ_TW;
constexpr size_t OFF_INST = OFF_TW64 + SZ_TW64;
constexpr size_t OFF_RT = OFF_INST + SZ_INST;
constexpr size_t OFF_CT = OFF_RT + SZ_RT;
constexpr size_t OFF_SUM = OFF_CT + SZ_CT;
constexpr size_t NA_BYTES = OFF_SUM + SZ_SUM;

// The scratch array itself.  Shared by every call on a device; it keeps the
// contents of the last call.
static __device__ __align__(256) unsigned char g_field_scratch[NA_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
// per device: the array's device address the twiddles were uploaded to, and
// the grid whose demag spectrum the array holds
struct DeviceState {
  unsigned char* base = nullptr;
  bool tensor_valid = false;
  int nx = 0, ny = 0;
  double dx = 0, dy = 0, dz = 0;
};
DeviceState g_state[kMaxDevices];

int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}
int log2_of(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// With the device current: resolve the array's device address; on the
// first call for this address fill the twiddle tables (synchronously) and
// forget any demag spectrum.  Caller holds g_setup_mutex.
llg_status setup_device(int dev, unsigned char** base, const char** msg) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_field_scratch);
  if (e != cudaSuccess || p == nullptr) {
    if (msg) *msg = "llg_field_noalloc: cudaGetSymbolAddress of the scratch array failed";
    return LLG_ECUDA;
  }
  unsigned char* b = static_cast<unsigned char*>(p);
  if (g_state[dev].base == b) {
    *base = b;
    return LLG_OK;
  }
  g_state[dev] = DeviceState{};
  static float2 htw[kTwiddleN];
  static double2 htw64[kTwiddleN];
  for (int k = 0; k < kTwiddleN; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)kTwiddleN;
    htw64[k] = make_double2(std::cos(ang), std::sin(ang));
    htw[k] = make_float2((float)htw64[k].x, (float)htw64[k].y);
  }
  if (cudaMemcpy(b + OFF_TW, htw, sizeof(htw), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b + OFF_TW64, htw64, sizeof(htw64), cudaMemcpyHostToDevice) != cudaSuccess) {
    if (msg) *msg = "llg_field_noalloc: uploading the twiddle tables failed";
    return LLG_ECUDA;
  }
  g_state[dev].base = b;
  *base = b;
  return LLG_OK;
}

// Writes the call's descriptor and its row and column tiles into the
// scratch; everything arrives as kernel arguments.
__global__ void noalloc_setup_kernel(DevInst d, int rows, int tx, DevInst* dI, RowTile* dRT, ColTile* dCT) {
  const int i = threadIdx.x;
  if (i == 0) *dI = d;
  const int nrt = (d.ny + rows - 1) / rows, nct = (d.Lx + tx - 1) / tx;
  if (i < nrt) dRT[i] = RowTile{0, 0, i * rows, min(rows, d.ny - i * rows), i};
  if (i < nct) dCT[i] = ColTile{0, i * tx, min(tx, d.Lx - i * tx), 0};
}
static_assert(NA_MAX_ROW_TILES <= 128 && NA_MAX_COL_TILES <= 128, "one set-up thread per tile");

}  // namespace

extern "C" llg_status llg_field_noalloc(const llg_problem* prob, const void* phi_dev, const void* m_dev,
                                        double t, int demag_only, void* B_dev, void* cuda_stream,
                                        const char** err_msg) {
  if (err_msg) *err_msg = "";
  if (!prob || !phi_dev || !m_dev || !B_dev) {
    if (err_msg) *err_msg = "llg_field_noalloc: prob, phi, m and B must not be NULL";
    return LLG_EINVAL;
  }
  const llg_problem& p = *prob;
  if (p.nz != 1 || p.nx < 4 || p.nx % 4 != 0 || p.nx > NA_MAX_N || p.ny < 1 || p.ny > NA_MAX_N) {
    if (err_msg)
      *err_msg = "llg_field_noalloc: grid exceeds the fixed scratch (needs nz == 1, nx a multiple of 4 "
                 "with 4 <= nx <= 128, 1 <= ny <= 128)";
    return LLG_EINVAL;
  }
  if (!(p.dx > 0 && p.dy > 0 && p.dz > 0 && p.Ms > 0 && p.A >= 0)) {
    if (err_msg) *err_msg = "llg_field_noalloc: dx, dy, dz, Ms must be > 0 and A >= 0";
    return LLG_EINVAL;
  }
  if ((((uintptr_t)m_dev) | ((uintptr_t)B_dev)) % 16 != 0) {
    if (err_msg) *err_msg = "llg_field_noalloc: m and B must be 16-byte aligned";
    return LLG_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    if (err_msg) *err_msg = "llg_field_noalloc: no usable current device";
    return LLG_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  unsigned char* base = nullptr;
  llg_status s = setup_device(dev, &base, err_msg);
  if (s != LLG_OK) return s;
  DeviceState& ds = g_state[dev];
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  // descriptor and work tiles of this call (same layout rules as llg_create)
  const int Px = std::max(16, pow2_at_least(2 * p.nx));
  const int Py = std::max(8, pow2_at_least(2 * p.ny));
  DevInst d;
  std::memset(&d, 0, sizeof d);
  d.nx = p.nx; d.ny = p.ny; d.nz = 1; d.Pz = 1;
  d.Lx = Px / 2; d.Py = Py;
  d.log2Lx = log2_of(d.Lx); d.log2Py = log2_of(Py);
  d.nodes = (long long)p.nx * p.ny;
  d.layer = d.nodes;
  d.Ms = p.Ms;
  d.cex_x = 2.0 * p.A / (p.Ms * p.dx * p.dx);
  d.cex_y = 2.0 * p.A / (p.Ms * p.dy * p.dy);
  d.cex_z = 2.0 * p.A / (p.Ms * p.dz * p.dz);
  d.kan = 2.0 * p.Ku / p.Ms;
  const double kn = std::sqrt(p.ku[0] * p.ku[0] + p.ku[1] * p.ku[1] + p.ku[2] * p.ku[2]);
  for (int c = 0; c < 3; ++c) {
    d.ku[c] = kn > 0 ? p.ku[c] / kn : 0.0;
    d.B_bias[c] = p.B_bias[c];
    d.rf_dir[c] = p.rf_dir[c];
  }
  for (int c = 0; c < 4; ++c) d.src[c] = p.src[c];
  d.b_rf = p.b_rf;
  d.f_rf = p.f_rf;
  d.sigmoid_a = p.sigmoid_a;
  d.alpha = p.alpha;
  d.alpha_edge = p.alpha_edge;
  d.absorb_nodes = p.absorb_nodes;
  d.absorb_x = p.absorb_x;
  d.absorb_y = p.absorb_y;
  d.V = p.dx * p.dy * p.dz;
  const int rows = rows_per_tile(d.Lx);
  const int nrt = (p.ny + rows - 1) / rows;
  d.ntile = nrt;
  d.tile_off = 0;
  const int tx = std::max(1, std::min(1024 / Py, d.Lx));
  const int nct = (d.Lx + tx - 1) / tx;

  DevInst* dI = reinterpret_cast<DevInst*>(base + OFF_INST);
  RowTile* dRT = reinterpret_cast<RowTile*>(base + OFF_RT);
  ColTile* dCT = reinterpret_cast<ColTile*>(base + OFF_CT);
  float* tens = reinterpret_cast<float*>(base + OFF_TENS);
  float2* spec = reinterpret_cast<float2*>(base + OFF_SPEC);
  float* psi = reinterpret_cast<float*>(base + OFF_PSI);
  float* dpsi = reinterpret_cast<float*>(base + OFF_DPSI);
  double* psitile = reinterpret_cast<double*>(base + OFF_SUM);
  double2* G = reinterpret_cast<double2*>(base + OFF_G);
  const float2* tw = reinterpret_cast<const float2*>(base + OFF_TW);
  const double2* tw64 = reinterpret_cast<const double2*>(base + OFF_TW64);

  fill_coef(d);
  noalloc_setup_kernel<<<1, 128, 0, st>>>(d, rows, tx, dI, dRT, dCT);
  cudaError_t e = cudaGetLastError();
  // the demag spectrum of this grid, FP64 on the device (G is cleared
  // inside), unless the array already holds it from the previous call
  const bool same = ds.tensor_valid && ds.nx == p.nx && ds.ny == p.ny && ds.dx == p.dx && ds.dy == p.dy &&
                    ds.dz == p.dz;
  if (e == cudaSuccess && !same) {
    ds.tensor_valid = false;
    e = build_tensor_spectrum<float>(tens, G, p.nx, p.ny, 1, Px, Py, 1, p.dx, p.dy, p.dz, tw64, st);
    if (e == cudaSuccess) {
      ds.tensor_valid = true;
      ds.nx = p.nx; ds.ny = p.ny;
      ds.dx = p.dx; ds.dy = p.dy; ds.dz = p.dz;
    }
  }
  if (e != cudaSuccess) {
    if (err_msg) *err_msg = "llg_field_noalloc: set-up kernel or tensor build failed";
    return LLG_ECUDA;
  }
  // psi from phi (the per-tile psi partials are not used by the field)
  launch_material_tiles<float>(dI, dRT, nrt, static_cast<const float*>(phi_dev), psi, dpsi, psitile, nullptr, st);

  RowArgs<float> a;
  std::memset(&a, 0, sizeof a);
  a.inst = dI;
  a.tiles = dRT;
  a.spec = spec;
  a.tw = tw;
  a.psi = psi;
  a.Yin = static_cast<const float*>(m_dev);
  // exchange scratch + twiddle table (W_{2Lx} for the row kernels, W_Py for
  // the column kernel): below the 48 KB default, no opt-in attribute needed
  const size_t smem_rows = (size_t)(kExch + 2 * d.Lx) * sizeof(float2);
  const size_t smem_cols = cols_smem_bytes<float>(Py);
  launch_rows<float>(a, ROW_FFT_ONLY, nrt, smem_rows, st, false);
  ColArgs<float> c;
  c.inst = dI;
  c.tiles = dCT;
  c.spec = spec;
  c.tw = tw;
  c.tens = tens;
  c.cols_max = tx;
  c.err = nullptr;
  launch_cols<float>(c, nct, smem_cols, st);
  a.Bout = static_cast<float*>(B_dev);
  a.t_field = t;
  a.demag_only = demag_only;
  launch_rows<float>(a, ROW_FIELD, nrt, smem_rows, st, false);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (err_msg) *err_msg = "llg_field_noalloc: kernel launch failed";
    return LLG_ECUDA;
  }
  return LLG_OK;
}
