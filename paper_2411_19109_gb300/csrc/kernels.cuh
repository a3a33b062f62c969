// Kernel argument blocks and launch helpers shared by kernels.cu and the
// host runtime.
#pragma once

#include "common.cuh"

namespace llg {

// Row-kernel modes.
enum RowMode : int {
  ROW_FFT_ONLY = 0,   // spectrum of M = Ms psi Yin (first stage of a step)
  ROW_STAGE = 1,      // demag inverse + field + RK4 stage + next-stage spectrum
  ROW_FIELD = 2,      // effective field (or demag only) of Yin -> Bout
  ROW_TERMINAL = 3,   // energies / lambda_N / explicit dJ/dpsi at m_N = Yin
  ROW_DP_STAGE = 4,   // demag inverse + field + Dormand-Prince stage + next-stage spectrum
  ROW_DP_START = 5,   // apply the last attempt's acceptance, first DP stage input + spectrum
};

template <typename T>
struct RowArgs {
  const DevInst* inst;
  const RowTile* tiles;
  cplx<T>* spec;
  const cplx<T>* tw;
  const T* psi;
  const T* Yin;       // stage input, read with halo
  const T* m;         // m_n, pointwise
  T* acc;             // RK accumulator
  T* Yout;            // next stage input (stages 1..3)
  T* mout;            // m_{n+1} (stage 4)
  T* Bout;            // recorded B_s (nullable) / field output (ROW_FIELD)
  T* ckpt;            // copy of m_{n+1} (stage 4, nullable)
  double* slots;      // objective slots (nullable: do not accumulate)
  double* pslots;     // spectral objective: per-(step, tile, box) port partials (nullable)
  const double* wtab; // spectral / curve objective: per-step adjoint weights
  const double* psimom;  // per row tile: sum psi x, sum psi y (curve objective's centre)
  const long long* step_base;
  int* err;           // error word (bounded waits that ran out)
  const double* rf;   // per instance, per step: b_rf sin(2 pi f t) at t = n dt + c dt, c = 0, 1/2, 1
  int local_step;
  int stage;          // 1..4
  int rows_max;       // smem sizing: rows per tile
  int demag_only;     // ROW_FIELD
  double t_field;     // ROW_FIELD time
  double dt;
  long long n_from;
  // Dormand-Prince stages (ROW_DP_STAGE, ROW_DP_START)
  const double* hst;  // per instance: t, h, last, done of the current attempt
  T* kbuf;            // slopes k_1..k_7, slot s-1 at kbuf + (s-1) * kstride
  long long kstride;  // 3 x all nodes
  T dpa[8];           // a(s+1, j), j = 1..s (stage s < 7); a(2, 1) for ROW_DP_START
  T dpe[8];           // b_j - b*_j, j = 1..7 (stage 7)
  double rtol, atol;  // error control (stage 7)
  double* eslots;     // per row tile: sum of the scaled squared errors (stage 7)
  const int* accept;  // ROW_DP_START: per instance, the last attempt was accepted
  const int* cnt;     // ROW_DP_START: per instance, accepted steps so far (checkpoint slot)
  T* ckall;           // ROW_DP_START: m of every ck_every-th accepted step k (slot k / ck_every at
                      // ckall + slot * kstride); nullable
  int ck_every;       // ROW_DP_START: checkpoint period in accepted steps (0 or 1: every step)
  const T* y5;        // ROW_DP_START: the last attempt's fifth-order solution
  // ROW_TERMINAL outputs
  T* lam;             // lambda_N
  T* psib;            // dJ/dpsi accumulator (sum)
  T* psic;            //                     (compensation)
  double* jterm;      // per-row-tile partial of the terminal J
  const double* psitile; // per-row-tile partial sums of psi
  long long nsteps;
};

template <typename T>
struct ColArgs {
  const DevInst* inst;
  const ColTile* tiles;
  cplx<T>* spec;
  const cplx<T>* tw;
  const T* tens;      // packed spectrum tables
  int cols_max;
  int* err;           // error word for bounded waits (nullable)
};

// Dynamic shared memory of the film column kernel for a column FFT of length
// Py: FFT groups (within kExch complex), W_Py, and the tensor records of the
// tile's 1024/Py columns plus the Nyquist column (4 components each).
template <typename T>
__host__ __device__ constexpr size_t cols_smem_bytes(int Py) {
  return (size_t)(kExch + Py) * sizeof(cplx<T>) + (size_t)(1024 / Py + 1) * (Py / 2 + 1) * 4 * sizeof(T);
}

// S: the real type of the adjoint's frequency domain (spectrum, twiddles and
// FFT arithmetic of the demag transpose): T itself, or dfloat for FP32 node
// arrays with a double-float spectrum.
template <typename T, typename S = T>
struct AdjArgs {
  const DevInst* inst;
  const RowTile* tiles;
  cplx<S>* spec;
  const cplx<S>* tw;
  const T* psi;
  const T* Ys;        // Y_s of this stage (halo)
  const T* Bbar;      // Bbar_s (halo)
  T* gpart;           // in: local part of g_s; out: local part of g_{s-1}
  T* lam;             // lambda_{n+1} (stage 1 writes lambda_n)
  T* G;               // running sum of g over the stages of the step
  T* psib;
  T* psic;
  const T* Yprev;     // Y and B of the next stage to be reversed
  const T* Bprev;
  T* BbarOut;
  const T* Dext;      // split adjoint stage: the demag transpose N * Bbar_s
                      // at the nodes, from its own row-transform launch
  const long long* step_base;
  int* err;
  int local_step;
  int stage;          // 4..1
  int seed_only;      // 1: only form u_4, Bbar_4 of step n from lambda
  int seed_next;      // stage 1: also seed step n-1 (Yprev/Bprev of its stage 4)
  const double* wtab; // spectral objective: per-step adjoint weights of the port boxes
  int rows_max;
  double dt;
  long long n_from;
  // Dormand-Prince adjoint stages (6..1)
  const double* hst;  // per instance: t, h of the step being reversed (h = 0: idle)
  T* ebuf;            // eta_1..eta_6 = (df/dY_s)^T kappa_s, slot s-1 at ebuf + (s-1) * kstride
  long long kstride;
  T dpb;              // b_{s-1} (b_6 for the seed)
  T dpa[8];           // dpa[i] = a(i, s-1), i = s..6
};

template <typename T>
void launch_rows(const RowArgs<T>& a, int mode, int ntiles, size_t smem, cudaStream_t st, bool z3);
// mb: the register-cap variant (blocks per SM it is compiled for; an
// unknown value takes the type's default)
template <typename T>
void launch_cols(const ColArgs<T>& a, int ntiles, size_t smem, cudaStream_t st, int mb = 0);
// film column pass with 16 register elements per lane (FP32, Py = 128, 256, 1024)
template <typename T>
void launch_cols16(const ColArgs<T>& a, int ntiles, size_t smem, cudaStream_t st);
template <typename T>
void smem_cols16(size_t smem);
__host__ __device__ constexpr bool cols16_length(int Py) { return Py == 128 || Py == 256 || Py == 1024; }
// column pass of 3D grids (nz > 1)
template <typename T>
void launch_cols3(const ColArgs<T>& a, int ntiles, size_t smem, cudaStream_t st);
template <typename T>
void smem_cols3(size_t smem);

// Columns per 3D column tile: enough (component, layer) sequences to fill the
// block with FFT groups, at least one column.
__host__ __device__ constexpr int cols3_per_tile(int Py, int nz, int Lx) {
  return (1024 / (Py * nz)) < 1 ? 1 : ((1024 / (Py * nz)) > Lx ? Lx : 1024 / (Py * nz));
}

// Sequence stride of the 3D column tile: one pad slot per 16 elements from
// Py = 128 up (the register FFTs' own exchange layout), made odd.
__host__ __device__ constexpr int cols3_stride(int L) { return row_padded_len(L) | 1; }

// Dynamic shared memory: 3 nz ncols sequences of cols3_stride(Py), W_Py^k
// for k < Py and W_Pz^k for k < 16.  In FP32 the largest tile (nz Py =
// 4096) takes 110 KB, so two blocks share an SM.
template <typename T>
__host__ __device__ constexpr size_t cols3_smem_bytes(int Py, int nz, int ncols) {
  return ((size_t)3 * nz * ncols * cols3_stride(Py) + Py + 16) * sizeof(cplx<T>);
}

template <typename T, typename S = T>
void launch_adj(const AdjArgs<T, S>& a, int ntiles, size_t smem, cudaStream_t st, bool z3, int mb = 0);

// Split adjoint stage (films): the node phase of adj_kernel with the demag
// transpose read from a.Dext and without the row transforms, whose own
// launches (spec_rows) run them in the frequency domain's type.
template <typename T>
void launch_adj_split(const AdjArgs<T>& a, int ntiles, size_t smem, cudaStream_t st, int mb);
template <typename T>
void smem_adj_split(size_t smem);
template <typename T>
__host__ __device__ constexpr size_t adj_split_smem_bytes(int L, int nx) {
  return (size_t)7 * (rows_per_tile(L) + 2) * nx * sizeof(T);
}

// Row transforms of a frequency domain of real type S for node arrays of
// type T, one row tile per block: DIR = +1 the inverse transform of the
// tile's spectrum rows to the field at the nodes (out), DIR = -1 the forward
// transform of the nodes' values (src) to the spectrum rows.
template <typename T, typename S>
struct SpecRowArgs {
  const DevInst* inst;
  const RowTile* tiles;
  cplx<S>* spec;
  const cplx<S>* tw;
  T* out;             // DIR = +1: [3][nodes] per instance (pooled like m)
  const T* src;       // DIR = -1: [3][nodes]
  int* err;
};
template <typename T, typename S>
void launch_spec_rows(const SpecRowArgs<T, S>& a, int dir, int ntiles, size_t smem, cudaStream_t st);
template <typename T, typename S>
void smem_spec_rows(size_t smem);
template <typename S>
__host__ __device__ constexpr size_t spec_rows_smem_bytes(int L) {
  return (size_t)(kExch + 2 * L + pass_tw_len<S>(L)) * sizeof(cplx<S>);
}
template <typename T, int MODE>
void launch_rows_mode(const RowArgs<T>& a, int ntiles, size_t smem, cudaStream_t st, bool z3);
template <typename T, int MODE>
void smem_rows_mode(size_t smem);
template <typename T>
void smem_cols(size_t smem);
template <typename T, typename S = T>
void smem_adj(size_t smem);
// Dormand-Prince adjoint stages, reverse-sweep gather, and step control
template <typename T>
void launch_adj_dp(const AdjArgs<T>& a, int ntiles, size_t smem, cudaStream_t st, bool z3);
template <typename T>
void smem_adj_dp(size_t smem);
template <typename T>
void launch_dp_gather(const DevInst* inst, const RowTile* tiles, int ntiles, const T* ckall, long long kstride,
                      const long long* slot, T* out, cudaStream_t st);
template <typename T>
void launch_dp_push(const DevInst* inst, const RowTile* tiles, int ntiles, const T* src, T* seg, long long kstride,
                    const long long* jptr, T* mrev, cudaStream_t st);
void launch_dp_control(const DevInst* inst, int n_inst, const double* eslots, double* hst, int* accept, int* cnt,
                       double* sched, long long max_steps, double T_end, int* overflow, cudaStream_t st);
// reverse index *rptr: each instance's step k = cnt - 1 - r with its (t, h)
// into hst and its state slot k - base[i] (base nullable: 0) into slot
void launch_dp_reverse_state(int n_inst, const double* sched, const int* cnt, const long long* rptr, double* hst,
                             long long* slot, const long long* base, cudaStream_t st);
// periodic checkpoints, reverse block b of K reverse indices: per instance
// the window's last step khi = cnt - 1 - b K, its first replayed step k0 (a
// checkpoint, k0 = K floor(max(0, cnt - (b + 1) K) / K)) and that
// checkpoint's slot (-1: the instance has no step in this block)
void launch_dp_replay_plan(int n_inst, const int* cnt, long long b, long long K, long long* k0, long long* khi,
                           long long* ckslot, cudaStream_t st);
// replay step *jptr of the block: instance i advances its step k0 + j with
// the recorded (t, h) while k0 + j < khi, else idles with h = 0
void launch_dp_replay_state(int n_inst, const double* sched, const long long* jptr, const long long* k0,
                            const long long* khi, double* hst, cudaStream_t st);
template <typename T>
void set_smem_limits(size_t stage, size_t misc, size_t cols, size_t adj);
template <typename T>
void launch_material_tiles(const DevInst* inst, const RowTile* tiles, int ntiles, const T* phi, T* psi,
                           T* dpsi, double* psitile, double* psimom, cudaStream_t st);
template <typename T>
void launch_grad_finish_tiles(const DevInst* inst, const RowTile* tiles, int ntiles, const T* dpsi,
                              const T* psib, const T* psic, const double* w, T* out, const T* lam, T* dm0,
                              cudaStream_t st);
template <typename T>
void launch_levelset_tiles(const DevInst* inst, const RowTile* tiles, int ntiles, T* phi, const T* grad,
                           const unsigned char* mask, double lr, unsigned int* maxbits, cudaStream_t st);
void launch_set_step(long long* step_base, long long v, cudaStream_t st);
void launch_port_series(const DevInst* inst, int n_inst, const double* pslots, const double* psitile,
                        long long nsteps1, double* P, cudaStream_t st);
void launch_reduce_slots(const DevInst* inst, int n_inst, const double* slots, long long nslots,
                         const double* jterm, const double* psitile, const double* psimom, double* J,
                         cudaStream_t st);
int rows_threads();
int cols_threads();
int adj_threads();

template <typename T>
cudaError_t build_tensor_spectrum(T* table, double2* G, int nx, int ny, int nz, int Px, int Py, int Pz,
                                  double dx, double dy, double dz, const double2* tw, cudaStream_t st);
long long tensor_table_len(int Px, int Py, int Pz);
long long tensor_scratch_len(int Px, int Py, int Pz);

}  // namespace llg
