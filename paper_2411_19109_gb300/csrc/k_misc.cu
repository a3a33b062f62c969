// Kernel-family dispatch and the small untemplated kernels.
#include "kernels.cuh"

namespace llg {

int rows_threads() { return 384; }
int cols_threads() { return 384; }
int adj_threads() { return 384; }

__global__ void set_step_kernel(long long* p, long long v) { *p = v; }

// J_i = Kahan sum of the per-(step, row tile) partials + terminal term + area
// penalty on the mean of psi.  Every sum runs in a fixed order, so J is
// reproducible bit for bit.
__global__ void reduce_slots_kernel(const DevInst* inst, const double* slots, long long nsteps1,
                                    const double* jterm, const double* psitile, const double* psimom, double* J) {
  __shared__ double red[32];
  const DevInst& I = inst[blockIdx.x];
  const long long nslots = nsteps1 * I.ntile;
  double sum = 0.0, comp = 0.0;
  for (long long k = threadIdx.x; k < nslots; k += blockDim.x) {
    const double y = slots[I.slot_off + k] - comp;
    const double t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  const double tot = block_sum(sum - comp, red);
  if (threadIdx.x == 0) {
    double j = tot, ps = 0.0;
    for (int t = 0; t < I.ntile; ++t) {
      j += jterm[I.tile_off + t];
      ps += psitile[I.tile_off + t];
    }
    if (I.objective == 1) {
      const double f = ps / (double)I.nodes - I.area_target;
      j += I.penalty_w * f * f;
    } else if (I.objective == 3) {
      // size and centre terms of Eq. 9 (the sampled curve is added on the host)
      double sx = 0.0, sy = 0.0;
      for (int t = 0; t < I.ntile; ++t) {
        sx += psimom[2 * (I.tile_off + t)];
        sy += psimom[2 * (I.tile_off + t) + 1];
      }
      const double f = ps / (double)I.nodes - I.area_target;
      j += I.penalty_w * f * f + I.centre_w * (fabs(sx / ps - I.centre_x0) + fabs(sy / ps - I.centre_y0));
    }
    J[blockIdx.x] = j;
  }
}

// Series of the spectral and curve objectives from the per-(step, tile,
// channel) partials, tiles added in order (block per instance).  Spectral:
// port-box means P_b[n] of m_comp (channel b).  Curve: P[n] = sum psi m_comp
// / sum psi in channel 0, sum psi in channel 1.
__global__ void port_series_kernel(const DevInst* inst, const double* pslots, const double* psitile,
                                   long long nsteps1, double* P) {
  const DevInst& I = inst[blockIdx.x];
  if (I.objective != 2 && I.objective != 3) return;
  double S = 0.0;
  if (I.objective == 3)
    for (int k = 0; k < I.ntile; ++k) S += psitile[I.tile_off + k];
  for (long long e = threadIdx.x; e < 2 * nsteps1; e += blockDim.x) {
    const long long n = e >> 1;
    const int b = (int)(e & 1);
    if (I.objective == 3) {
      double s = 0.0;
      if (b == 0)
        for (int k = 0; k < I.ntile; ++k) s += pslots[2 * (I.slot_off + n * I.ntile + k)];
      P[I.wt_off + e] = b == 0 ? s / S : S;
      continue;
    }
    const long long cnt = (long long)(I.boxes[b][1] - I.boxes[b][0]) * (I.boxes[b][3] - I.boxes[b][2]) * I.nz;
    double s = 0.0;
    for (int k = 0; k < I.ntile; ++k) s += pslots[2 * (I.slot_off + n * I.ntile + k) + b];
    P[I.wt_off + e] = cnt > 0 ? s / (double)cnt : 0.0;
  }
}

void launch_port_series(const DevInst* inst, int n_inst, const double* pslots, const double* psitile,
                        long long nsteps1, double* P, cudaStream_t st) {
  port_series_kernel<<<n_inst, 256, 0, st>>>(inst, pslots, psitile, nsteps1, P);
}

void launch_set_step(long long* step_base, long long v, cudaStream_t st) {
  set_step_kernel<<<1, 1, 0, st>>>(step_base, v);
}

void launch_reduce_slots(const DevInst* inst, int n_inst, const double* slots, long long nsteps1,
                         const double* jterm, const double* psitile, const double* psimom, double* J,
                         cudaStream_t st) {
  reduce_slots_kernel<<<n_inst, 256, 0, st>>>(inst, slots, nsteps1, jterm, psitile, psimom, J);
}

template <typename T>
void launch_rows(const RowArgs<T>& a, int mode, int ntiles, size_t smem, cudaStream_t st, bool z3) {
  switch (mode) {
    case ROW_FFT_ONLY: launch_rows_mode<T, ROW_FFT_ONLY>(a, ntiles, smem, st, z3); break;
    case ROW_STAGE: launch_rows_mode<T, ROW_STAGE>(a, ntiles, smem, st, z3); break;
    case ROW_FIELD: launch_rows_mode<T, ROW_FIELD>(a, ntiles, smem, st, z3); break;
    case ROW_DP_STAGE: launch_rows_mode<T, ROW_DP_STAGE>(a, ntiles, smem, st, z3); break;
    case ROW_DP_START: launch_rows_mode<T, ROW_DP_START>(a, ntiles, smem, st, z3); break;
    default: launch_rows_mode<T, ROW_TERMINAL>(a, ntiles, smem, st, z3); break;
  }
}

// Step control of the Dormand-Prince integrator, one block per instance:
// err = sqrt(mean of the scaled squared errors of the attempt) from the
// per-tile sums (added in a fixed order); accept if err <= 1 (then the step
// (t, h) goes to the schedule, t advances, exactly to T_end on the last
// step); h <- h min(5, max(0.2, 0.9 err^(-1/5))), shortened to end at T_end.
// hst per instance: t, h, last (this attempt ends at T_end), done.
__global__ void dp_control_kernel(const DevInst* inst, const double* eslots, double* hst, int* accept, int* cnt,
                                  double* sched, long long max_steps, double T_end, int* overflow) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  const DevInst& I = inst[i];
  double v = 0.0;
  for (int k = threadIdx.x; k < I.ntile; k += blockDim.x) v += eslots[I.tile_off + k];
  const double S = block_sum(v, red);
  if (threadIdx.x != 0) return;
  double* H = hst + 4 * i;
  if (H[3] != 0.0) {
    accept[i] = 0;
    return;
  }
  const double err = sqrt(S / (3.0 * (double)I.nodes));
  const bool ok = err <= 1.0;
  double t = H[0], h = H[1];
  if (ok) {
    const long long k = cnt[i];
    if (k >= max_steps) {
      *overflow = 1;
      H[1] = 0.0;
      H[3] = 1.0;
      accept[i] = 0;
      return;
    }
    sched[2 * (k * gridDim.x + i)] = t;
    sched[2 * (k * gridDim.x + i) + 1] = h;
    cnt[i] = (int)(k + 1);
    t = H[2] != 0.0 ? T_end : t + h;
  }
  const double fac = err == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2)));
  h *= fac;
  if (ok && H[2] != 0.0) {
    h = 0.0;
    H[2] = 0.0;
    H[3] = 1.0;
  } else {
    const bool last = h >= T_end - t;
    if (last) h = T_end - t;
    H[2] = last ? 1.0 : 0.0;
  }
  H[0] = t;
  H[1] = h;
  accept[i] = ok ? 1 : 0;
}

void launch_dp_control(const DevInst* inst, int n_inst, const double* eslots, double* hst, int* accept, int* cnt,
                       double* sched, long long max_steps, double T_end, int* overflow, cudaStream_t st) {
  dp_control_kernel<<<n_inst, 256, 0, st>>>(inst, eslots, hst, accept, cnt, sched, max_steps, T_end, overflow);
}

// Reverse step r of the adjoint sweep: each instance reverses its accepted
// step k = cnt - 1 - r with the recorded (t_k, h_k), or idles (h = 0).
__global__ void dp_reverse_state_kernel(int n_inst, const double* sched, const int* cnt, const long long* rptr,
                                        double* hst, long long* slot, const long long* base) {
  const long long r = *rptr;
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    const long long k = (long long)cnt[i] - 1 - r;
    if (k >= 0) {
      hst[4 * i] = sched[2 * (k * n_inst + i)];
      hst[4 * i + 1] = sched[2 * (k * n_inst + i) + 1];
      slot[i] = k - (base ? base[i] : 0);
    } else {
      hst[4 * i] = 0.0;
      hst[4 * i + 1] = 0.0;
      slot[i] = -1;
    }
  }
}

void launch_dp_reverse_state(int n_inst, const double* sched, const int* cnt, const long long* rptr, double* hst,
                             long long* slot, const long long* base, cudaStream_t st) {
  dp_reverse_state_kernel<<<1, 256, 0, st>>>(n_inst, sched, cnt, rptr, hst, slot, base);
}

__global__ void dp_replay_plan_kernel(int n_inst, const int* cnt, long long b, long long K, long long* k0,
                                      long long* khi, long long* ckslot) {
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    const long long hi = (long long)cnt[i] - 1 - b * K;
    if (hi < 0) {
      k0[i] = 0;
      khi[i] = 0;
      ckslot[i] = -1;
      continue;
    }
    const long long lo = max(0LL, (long long)cnt[i] - (b + 1) * K);
    k0[i] = (lo / K) * K;
    khi[i] = hi;
    ckslot[i] = lo / K;
  }
}
void launch_dp_replay_plan(int n_inst, const int* cnt, long long b, long long K, long long* k0, long long* khi,
                           long long* ckslot, cudaStream_t st) {
  dp_replay_plan_kernel<<<1, 256, 0, st>>>(n_inst, cnt, b, K, k0, khi, ckslot);
}

__global__ void dp_replay_state_kernel(int n_inst, const double* sched, const long long* jptr, const long long* k0,
                                       const long long* khi, double* hst) {
  const long long j = *jptr;
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    const long long k = k0[i] + j;
    if (k < khi[i]) {
      hst[4 * i] = sched[2 * (k * n_inst + i)];
      hst[4 * i + 1] = sched[2 * (k * n_inst + i) + 1];
    } else {
      hst[4 * i] = 0.0;
      hst[4 * i + 1] = 0.0;
    }
  }
}
void launch_dp_replay_state(int n_inst, const double* sched, const long long* jptr, const long long* k0,
                            const long long* khi, double* hst, cudaStream_t st) {
  dp_replay_state_kernel<<<1, 256, 0, st>>>(n_inst, sched, jptr, k0, khi, hst);
}

template <typename T>
void set_smem_limits(size_t stage, size_t misc, size_t cols, size_t adj) {
  smem_rows_mode<T, ROW_FFT_ONLY>(misc);
  smem_rows_mode<T, ROW_STAGE>(stage);
  smem_rows_mode<T, ROW_FIELD>(misc);
  smem_rows_mode<T, ROW_TERMINAL>(misc);
  smem_cols<T>(cols);
  smem_adj<T>(adj);
  smem_rows_mode<T, ROW_DP_STAGE>(stage);
  smem_rows_mode<T, ROW_DP_START>(misc);
  smem_adj_dp<T>(adj);
}

template void launch_rows<float>(const RowArgs<float>&, int, int, size_t, cudaStream_t, bool);
template void launch_rows<double>(const RowArgs<double>&, int, int, size_t, cudaStream_t, bool);
template void set_smem_limits<float>(size_t, size_t, size_t, size_t);
template void set_smem_limits<double>(size_t, size_t, size_t, size_t);

}  // namespace llg
