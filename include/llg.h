/*
 * llg.h -- C ABI of the GB300 level-set / adjoint LLG solver.
 *
 * The library integrates the Landau-Lifshitz-Gilbert equation (Eq. 11 of
 * arXiv:2411.19109, Methods) on a nodal finite-difference grid for a batch of
 * independent instances, evaluates an objective J per instance and returns
 * dJ/dPhi, the gradient with respect to the level-set function Phi (Eq. 1)
 * through the material map psi = 1/(1 + exp(-a Phi)) (Eq. 4), by the discrete
 * adjoint of the time stepper (the adjoint-state system, Eq. 6, and the
 * parameter integral, Eq. 7, taken through the RK4 stages).  levelset_step
 * applies the gradient-descent update (Eq. 5) on Phi and renormalises Phi to
 * [-1, 1] (Results, "Level-set method").
 *
 * Discretisation (shared with the FP64 oracle used by the tests):
 *   node i owns a cuboid dx*dy*dz; Ms_i = Ms psi_i, A_i = A psi_i;
 *   B_ex,i = (2A/Ms) sum_j w_ij (m_j - m_i)/h^2, w_ij = 2 psi_j/(psi_i + psi_j)
 *            (harmonic-mean edge coupling, free boundaries);
 *   B_an   = (2 Ku/Ms)(m.u)u;  B_z = B_bias + b_rf sin(2 pi f t) e_rf on src;
 *   B_d    = -mu0 N * (Ms psi m), N the cell-averaged (Newell) tensor,
 *            evaluated by zero-padded FFT convolution (padded extents
 *            Px, Py from llg_padded_extents; Pz = 1 for a film, else the
 *            power of two >= 2 nz: 6 tensor components);
 *   dm/dt  = -gamma/(1+alpha_i^2) [m x B + alpha_i m x (m x B)];
 *   classic RK4 at fixed dt, t_n = n dt, no renormalisation of m.
 *
 * Memory and ownership.  Every *_dev pointer is device memory owned by the
 * caller; instances are packed back to back in the order given to
 * llg_create.  Per instance i with nodes n_i = nx*ny*nz:
 *   phi, grad  [n_i]          layout [z][y][x], x fastest
 *   m0, mT     [3][n_i]       layout [component][z][y][x]
 *   mask       [n_i] uint8    1 = design region
 * Element type: float for LLG_FP32, double for LLG_FP64 (llg_options).
 * The library owns its scratch (spectra, tensors, checkpoints, stage
 * records); it allocates them in llg_create and frees them in llg_destroy.
 *
 * Streams.  All work runs on the stream given to llg_create.  llg_forward
 * and llg_adjoint synchronise that stream before they return (they copy J
 * and the device error word to the host); levelset_step and llg_field
 * return as soon as the work is queued.  With llg_options.use_graph the
 * RK4 segments are replayed from CUDA graphs captured on a private stream
 * of the context (once per segment kind and length) and launched on the
 * context's stream, so the caller's stream may be the legacy default one.
 *
 * Errors.  Functions return llg_status; no exception crosses the ABI.  On a
 * non-OK status llg_last_error(ctx) holds a one-line description.  A device
 * wait that exceeds its bound returns LLG_ETIMEOUT; a non-finite J returns
 * LLG_ENONFINITE (the outputs are still written).
 */
#ifndef LLG_H
#define LLG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LLG_OK = 0,
  LLG_EINVAL = 1,     /* invalid argument or unsupported problem size        */
  LLG_ENOMEM = 2,     /* device allocation failed                            */
  LLG_ECUDA = 3,      /* a CUDA runtime call failed                          */
  LLG_ETIMEOUT = 4,   /* a bounded device wait ran out                       */
  LLG_ENONFINITE = 5, /* J is NaN or Inf                                     */
  LLG_ESTATE = 6      /* call order violated (adjoint without forward, ...)  */
} llg_status;

enum { LLG_J_PORT = 0, LLG_J_ENERGY_AREA = 1, LLG_J_SPECTRAL = 2, LLG_J_CURVE = 3 };
enum { LLG_FP32 = 0, LLG_FP64 = 1 };
enum { LLG_CKPT_STORE_ALL = 0, LLG_CKPT_PERIODIC = 1, LLG_CKPT_BINOMIAL = 2 };
enum { LLG_INT_RK4 = 0, LLG_INT_DOPRI5 = 1 };
enum { LLG_SPEC_WORKING = 0, LLG_SPEC_DFLOAT = 1 };
enum { LLG_TUNE_DEFAULT = 0, LLG_TUNE_MEASURE = 1, LLG_TUNE_GIVEN = 2 };
enum { LLG_RECORD_STAGES = 0, LLG_RECORD_STATES = 1 };

/* Launch configuration of the hot kernels: which compiled variant of a
 * kernel family runs and how the batch is split over streams.  Only
 * col_lanes changes results (a different FFT radix order in the FP32
 * column pass, so FP32 rounding differs); the others are bit-identical.
 * Fields that do not apply to a context (col_lanes in FP64, the
 * double-float fields without LLG_SPEC_DFLOAT) are ignored. */
typedef struct {
  int col_lanes;   /* FP32 film column pass at 128-, 256- and 1024-point
                      columns: 16 (16-element FFT lanes, 192-thread blocks,
                      one shared-memory exchange fewer) or 8 (8-element
                      lanes, 384-thread blocks)                           */
  int col_blocks;  /* double-float column pass: the blocks per SM its
                      register cap is compiled for, 2 (80 registers) or 1  */
  int adj_blocks;  /* double-float adjoint stage: blocks per SM the fused
                      kernel (1 or 2) or the split stage's FP32 node phase
                      (2, or 3 with a 56-register cap and spills; 1 acts
                      as 2) is compiled for                               */
  int groups;      /* RK4 segments as 2 independent chains (even and odd
                      instances on two streams) or 1                      */
  int adj_split;   /* double-float adjoint stage: 1 = three launches (the
                      inverse row transform to a field buffer, the FP32
                      node phase at 2 blocks per SM, the forward row
                      transform), 0 = one fused kernel (its FFT registers
                      allow one block per SM)                             */
} llg_launch;

/* One instance.  SI units (m, A/m, J/m, J/m^3, T, Hz, s). */
typedef struct {
  int nx, ny, nz;            /* nodes; nx % 4 == 0, 4 <= nx <= 1024 (FP64:
                                780), 1 <= ny <= 512, 1 <= nz <= 8 (1 = film)  */
  double dx, dy, dz;         /* node spacing = cell size                       */
  double Ms, A, Ku;          /* saturation magnetisation, exchange, anisotropy */
  double ku[3];              /* anisotropy axis (normalised by the library)    */
  double alpha, alpha_edge;  /* Gilbert damping; value at an absorbing edge    */
  int absorb_nodes;          /* ramp width W (0 = none): alpha_i = alpha +
                                (alpha_edge - alpha) max(0, (W - d_i)/W)       */
  int absorb_x, absorb_y;    /* which pairs of edges absorb                   */
  double B_bias[3];          /* static field                                   */
  double b_rf, f_rf;         /* RF amplitude and frequency                     */
  double rf_dir[3];          /* RF direction                                   */
  int src[4];                /* RF source box x0,x1,y0,y1 (half open; boxes span
                                every z layer)                                 */
  double dt;                 /* time step                                      */
  long long nsteps;          /* number of RK4 steps N                          */
  double sigmoid_a;          /* a of Eq. 4                                     */
  int objective;             /* LLG_J_PORT, LLG_J_ENERGY_AREA, LLG_J_SPECTRAL, LLG_J_CURVE */
  int comp, power;           /* LLG_J_PORT: sampled component, exponent 1 or 2 */
  int boxes[2][4];           /* LLG_J_PORT: boxes x0,x1,y0,y1                   */
  double weights[2];         /* LLG_J_PORT: J = sum_{n>=n_from} sum_b w_b
                                mean_{box b}(m_comp,n ^ power)                 */
  long long n_from;          /* first step index in the running sum            */
  double area_target;        /* LLG_J_ENERGY_AREA: J = (E_d + E_ex)(m_N) /
                                (mu0 Ms^2/2 * V_domain) + penalty_w *
                                (mean(psi) - area_target)^2  (Eq. 9 size term) */
  double penalty_w;
  int nfreq;                 /* LLG_J_SPECTRAL: J = sum_b w_b sum_q |X_b(f_q)|,
                                X_b(f) = sum_{n >= n_from} P_b[n] exp(-2 pi i f n dt),
                                P_b[n] = mean_{box b} m_comp,n (Eq. 10: port
                                spectra summed over a frequency window, taken
                                at the window's frequencies); 1 <= nfreq <= 8,
                                n_from >= 1                                  */
  double freqs[8];           /* LLG_J_SPECTRAL: the frequencies f_q (Hz)     */
  const double* drive;       /* optional host table of the applied drive b at
                                t = n dt + c dt, c = 0, 1/2, 1, for n = 0..nsteps
                                (3 nsteps + 3 values, tesla, index 3n + 2c),
                                applied on the source box along rf_dir in place
                                of b_rf sin(2 pi f_rf t); NULL: the sine.  Read
                                at llg_create only.  llg_field ignores it (its
                                time argument is not a stage time).          */
  int nsample;               /* LLG_J_CURVE: J = sum_j w_j |P(m_{n_j}) - T_j|
                                + penalty_w (mean psi - area_target)^2
                                + centre_w (|x_c - x_0| + |y_c - y_0|), with
                                P = sum psi m_comp / sum psi (Eq. 8 sampled at
                                the end of each field level) and (x_c, y_c) the
                                psi-weighted mean node index (x, y) (Eq. 9);
                                nsample >= 1                                 */
  const long long* sample_step;  /* LLG_J_CURVE: host array [nsample] of steps
                                n_j, strictly increasing, 1 <= n_j <= nsteps;
                                the three sample arrays are read at llg_create
                                only                                         */
  const double* sample_target;   /* LLG_J_CURVE: host array [nsample], T_j    */
  const double* sample_weight;   /* LLG_J_CURVE: host array [nsample], w_j    */
  double centre_w;           /* LLG_J_CURVE: weight of the centre term        */
  double centre_target[2];   /* LLG_J_CURVE: (x_0, y_0), node-index units     */
} llg_problem;

typedef struct {
  int precision;   /* LLG_FP32 or LLG_FP64                                     */
  int ckpt;        /* LLG_CKPT_PERIODIC (O(sqrt N) memory), LLG_CKPT_STORE_ALL,
                      or LLG_CKPT_BINOMIAL (seg_len + 1 stored states, each
                      step advanced at most r + 1 times, r the smallest
                      with C(seg_len + r, r) >= nsteps)                      */
  int seg_len;     /* periodic: segment length K; binomial: free snapshot
                      slots s; 0 = ceil(sqrt(nsteps)) for both               */
  int use_graph;   /* 1 = replay captured CUDA graphs of whole segments
                      (ignored while time_kernels = 1)                        */
  int tune;        /* launch configuration (llg_launch): LLG_TUNE_DEFAULT
                      {16, 2, 2, 2, 1}; LLG_TUNE_MEASURE: llg_create times each
                      field's candidates on this batch (the kernel families
                      they change, a few ms) and keeps the fastest, cached
                      per device and batch shape for the process;
                      LLG_TUNE_GIVEN: `launch` below as given             */
  int time_kernels;/* 1 = bracket every stage-kernel launch with CUDA events    */
  int integrator;  /* LLG_INT_RK4: fixed step dt for nsteps steps.
                      LLG_INT_DOPRI5: adaptive step size (Methods), the
                      Dormand-Prince 5(4) pair from t = 0 to T = nsteps * dt
                      with initial step dt; each instance has its own step
                      size: err = sqrt(mean((psi e / (atol + rtol max(|psi
                      m|, |psi y5|)))^2)) over nodes and components, accept
                      if err <= 1, h <- h min(5, max(0.2, 0.9 err^-1/5)),
                      the last step shortened to end at T.  At most
                      seg_len (0: nsteps) accepted steps and 4 nsteps
                      attempts per instance (LLG_ETIMEOUT beyond).  The
                      gradient is the exact derivative over the accepted
                      steps (their sizes held fixed).  Checkpoints:
                      LLG_CKPT_STORE_ALL keeps m of every accepted step;
                      otherwise m of every K-th accepted step, K =
                      ceil(sqrt(seg_len or nsteps)), and the reverse sweep,
                      in blocks of K steps, first replays each instance's
                      recorded steps (t_k, h_k) from the checkpoint at or
                      before its block (bit-identical states; up to 2K - 1
                      replayed steps per block).  Needs the
                      LLG_J_ENERGY_AREA objective and the sine drive (no
                      drive table); use_graph replays captured attempts.   */
  double rtol, atol; /* LLG_INT_DOPRI5 tolerances                            */
  int adj_spectral;  /* frequency domain of the adjoint's demag transpose
                        (the row and column FFTs, the stored spectrum and the
                        tensor spectrum it is multiplied by):
                        LLG_SPEC_WORKING in the working precision;
                        LLG_SPEC_DFLOAT (FP32 contexts, films, RK4) in
                        double-float, hi + lo FP32 pairs (about 48 bits),
                        while the node arrays stay FP32.  FP32 rounding of a
                        Fourier coefficient perturbs the transform at every
                        node by about 1e-7 of the whole field's norm, which
                        drowns the adjoint field far from where the
                        objective excites it (the design region between the
                        demultiplexer's ports and its source); double-float
                        brings that to about 1e-14.  The forward pass and
                        the per-node arithmetic are unchanged.              */
  llg_launch launch; /* LLG_TUNE_GIVEN: the configuration to use          */
  int record;        /* what a checkpoint segment keeps for the reverse
                        sweep (RK4): LLG_RECORD_STAGES every step's four
                        stage inputs and fields (8 arrays of 3 x nodes per
                        step), recorded once; LLG_RECORD_STATES only m per
                        step (one array per step), each reverse step
                        recomputing its four stages first (one more forward
                        step per step: less memory, more time).  Results are
                        bit-identical.                                      */
} llg_options;

typedef struct llg_ctx llg_ctx;

/* Set up the problem of the Methods section for `n_inst` instances: the
 * material map of Eq. 4, the effective field of Eq. 11 (exchange, anisotropy,
 * Zeeman, demag) and the objective.  Validates the problems, builds the
 * per-shape demag spectra (FP64 on the device, stored in the working
 * precision, and in double-float for LLG_SPEC_DFLOAT), allocates all scratch
 * and fixes the launch configuration (llg_options.tune; llg_launch_config
 * reports it).  `cuda_stream` is a cudaStream_t (NULL = default stream).
 * Every instance must have the same nsteps, n_from and dt.
 * Returns LLG_EINVAL for unsupported sizes (nx % 4 != 0, nx outside [4, 1024],
 * ny outside [1, 512], nz outside [1, 8], or a row or column tile that does
 * not fit in shared memory: the adjoint's row tile stages 7 node arrays over
 * 3 rows, so nx <= 780 in FP64 (any allowed nx in FP32); a 3D grid's column
 * tile holds all nz layers of one padded column, so nz * Py <= 4096 in FP32
 * and <= 2048 in FP64, Py the padded y extent), and LLG_ENOMEM if the scratch
 * does not fit. */
llg_status llg_create(const llg_problem* inst, int n_inst, const llg_options* opt,
                      void* cuda_stream, llg_ctx** out);

/* Forward pass (Eq. 4, then Eq. 11 integrated by RK4, and the objective:
 * the port functional, Eq. 9's energy and size terms, Eq. 10's spectral
 * sum or Eq. 8's magnetisation curve): psi from phi, nsteps from m0, J per
 * instance.
 * J_host: [n_inst] doubles (required).  mT_dev: final m (nullable).
 * Keeps the checkpoints that llg_adjoint needs. */
llg_status llg_forward(llg_ctx* ctx, const void* phi_dev, const void* m0_dev,
                       double* J_host, void* mT_dev);

/* LLG_INT_DOPRI5: the accepted steps (t_k, h_k) of instance `inst` in the
 * last llg_forward, up to `cap` of them into the host arrays t_host, h_host;
 * *count receives the number of accepted steps.  LLG_ESTATE without a
 * forward pass or for the RK4 integrator, LLG_EINVAL for a bad instance. */
llg_status llg_adaptive_steps(llg_ctx* ctx, int inst, double* t_host, double* h_host, long long cap,
                              long long* count);

/* Reverse sweep after llg_forward on the same inputs: the adjoint-state
 * recursion (Eq. 6) and the parameter integral (Eq. 7) in their exact
 * discrete form through the RK4 stages, then dJ/dPhi = a psi (1 - psi) dJ/dpsi
 * (Eq. 4).  Writes dJ/dPhi (all nodes, unmasked) to dJdphi_dev and, if
 * non-NULL, dJ/dm0 to dJdm0_dev.  dJ_dextra (nullable, n_inst host doubles):
 * the cotangent of each instance's J under a combination made outside the
 * library (e.g. Eq. 10 as the sum of the two frequency runs of a candidate,
 * or an autograd graph above J); the outputs are then the gradients of
 * sum_i dJ_dextra[i] J_i, instance by instance.  NULL means 1 for every
 * instance.  LLG_ESTATE if no forward pass precedes it, LLG_EINVAL for a
 * non-finite dJ_dextra. */
llg_status llg_adjoint(llg_ctx* ctx, const double* dJ_dextra, void* dJdphi_dev, void* dJdm0_dev);

/* Level-set update (Eq. 5, and the renormalisation of the Results section's
 * level-set method) on the design mask, Phi <- Phi - lr grad, then Phi <- Phi / max|Phi|
 * over the mask, per instance (an instance whose masked max is 0 is left
 * unscaled).  Nodes outside the mask are not touched. */
llg_status levelset_step(llg_ctx* ctx, void* phi_dev, const void* grad_dev,
                         const unsigned char* mask_dev, double lr);

/* Effective field B (tesla) of Eq. 11 (Methods: exchange, anisotropy,
 * Zeeman, demag) of the magnetisation m_dev at time t for all instances,
 * psi taken from phi_dev (Eq. 4); demag_only != 0 returns B_d alone.
 * Layout of m_dev and B_dev as m0.  Diagnostic entry point for parity tests. */
llg_status llg_field(llg_ctx* ctx, const void* phi_dev, const void* m_dev, double t,
                     int demag_only, void* B_dev);

/* The launch configuration the context runs (llg_options.tune), and the
 * host time (ms) llg_create spent timing candidates (0 if none). */
llg_status llg_launch_config(llg_ctx* ctx, llg_launch* out, double* tune_ms);

/* Bytes the context holds on the device, and the device time (ms) of the last
 * llg_forward / llg_adjoint call.  (This and the calls below up to
 * llg_destroy are measurement and housekeeping; the paper has no
 * counterpart.) */
llg_status llg_query(llg_ctx* ctx, size_t* device_bytes, double* last_ms);

/* Number of kernels the context has launched since llg_create. */
long long llg_launch_count(llg_ctx* ctx);

/* Device time of one kernel family since llg_create, summed over CUDA-event
 * pairs recorded around each launch on the context's stream (needs
 * llg_options.time_kernels = 1; otherwise both outputs are 0).
 * family: 0 = forward row/stage kernel, 1 = column (demag) kernel in the
 *         working precision, 2 = adjoint stage kernel, 3 = column kernel of
 *         the adjoint's double-float frequency domain, 4 = row transforms
 *         of that domain (split adjoint stage; family 2 is then its FP32
 *         node phase). */
llg_status llg_kernel_time(llg_ctx* ctx, int family, long long* launches, double* total_ms);

const char* llg_last_error(llg_ctx* ctx);
void llg_destroy(llg_ctx* ctx);

/* Effective field of one FP32 instance without any device allocation.
 * There is no counterpart in the paper.  It serves callers that cannot
 * allocate device memory where they need a field evaluation: a host
 * application or framework that owns all device memory through its own
 * allocator and budget, or a latency-critical loop where cudaMalloc/cudaFree
 * would synchronise the device and stall other streams.
 * Same result as llg_field for a single instance, FP32 only (the 8-element
 * column kernel at every column length).
 * prob: the instance (nsteps, objective fields are ignored); phi_dev [ny*nx],
 * m_dev [3][ny][nx] and B_dev [3][ny][nx] are caller-owned float device
 * buffers (m_dev and B_dev 16-byte aligned); cuda_stream is a cudaStream_t
 * (NULL = default stream); the work is queued asynchronously on it.
 * Scratch: one fixed device array of about 5.3 MB inside this library, held
 * by every GPU that loads the library until the process exits.  It limits the
 * grid to nz == 1, nx a multiple of 4 with 4 <= nx <= 128 and 1 <= ny <= 128;
 * larger grids return LLG_EINVAL.  No cudaMalloc, cudaFree or allocating
 * library call is made; the call's descriptor and work tiles reach the
 * device as kernel arguments.  The first call on a device (with that device
 * current) looks up the array's device address and uploads constant tables,
 * synchronously: make that first call before any stream capture.  The demag
 * spectrum (FP64 set-up kernels) is rebuilt only when the grid or cell size
 * differs from the previous call's on that device.  All calls on a device
 * share the array and leave their contents in it; calls that overlap on the
 * GPU (different streams, no ordering) race with each other.  A device reset
 * is not supported: the host-side record of what the array holds would be
 * stale.  On error *err_msg (if non-NULL) points to a static description. */
llg_status llg_field_noalloc(const llg_problem* prob, const void* phi_dev, const void* m_dev, double t,
                             int demag_only, void* B_dev, void* cuda_stream, const char** err_msg);

/* FP64 fused multiply-add throughput of the current device (TFLOP/s), the
 * denominator of the FP64 path's arithmetic roofline.  There is no
 * counterpart in the paper: it is a measurement helper.  Runs 6 launches of
 * an FMA-chain kernel (8 chains x `iters` iterations per thread, 8 blocks of
 * 256 threads per SM) on cuda_stream and synchronises; the best of the last
 * four gives *tflops (and its duration in *ms, if non-NULL).  Allocates and
 * frees a small output buffer.  LLG_EINVAL for iters < 1 or tflops NULL,
 * LLG_ENOMEM / LLG_ECUDA on CUDA failures. */
llg_status llg_fp64_fma_rate(int iters, double* tflops, double* ms, void* cuda_stream);

/* ------------------------------------------------------------------------
 * RBF parameterisation of the level-set function and the optimiser step.
 * Phi on a rectangular design box is built from nrx*nry multiquadric cones
 * g_k(x) = s_k - sqrt(|x - x_k|^2 + c^2) (Eq. 2; centres at the centres of
 * equal cells of the box, c = the centre spacing), combined by the p-norm of
 * Eq. 3, F = ||g + dphi||_p - dphi with dphi = |min over RBFs and design
 * nodes of g|, and renormalised, Phi = F / max_design |F| (Results, "Level-
 * set method": Phi kept in [-1, 1]).  The amplitudes s (n = nrx*nry
 * doubles, k = iy*nrx + ix) are what the optimiser updates (Adam, Methods).
 * All three calls are asynchronous on the given stream and allocate
 * nothing; they return LLG_EINVAL for invalid arguments (checked before any
 * device work) and LLG_ECUDA if a launch fails.
 * ------------------------------------------------------------------------ */
typedef struct {
  int nx, ny;       /* grid of the phi array ([ny][nx], one layer)           */
  double dx, dy;    /* node spacing                                          */
  int box[4];       /* design box x0, x1, y0, y1 (node indices, half open)   */
  int nrx, nry;     /* RBF centres per axis                                  */
  double p;         /* p-norm exponent (the paper uses 90)                   */
} llg_rbf;

/* Bytes of device workspace llg_rbf_phi / llg_rbf_grad need (0 if r is
 * invalid): about 32 bytes per design node plus 16 per RBF. */
size_t llg_rbf_workspace_bytes(const llg_rbf* r);

/* Phi = F / max|F| on the design nodes of phi_dev ([ny][nx], float for
 * LLG_FP32, double for LLG_FP64); nodes outside the box are not touched.
 * s_dev: n amplitudes (double); work_dev: llg_rbf_workspace_bytes(r) bytes. */
llg_status llg_rbf_phi(const llg_rbf* r, const double* s_dev, void* phi_dev, int precision, void* work_dev,
                       void* cuda_stream);

/* dJ/ds (n doubles) for dJ/dPhi given in dJdphi_dev ([ny][nx], only design
 * nodes read): the exact derivative of the map above, through the shift and
 * the renormalisation (taken at the minimising node/RBF pair and the
 * maximising node, the first in index order on ties). */
llg_status llg_rbf_grad(const llg_rbf* r, const double* s_dev, const void* dJdphi_dev, int precision,
                        double* dJds_dev, void* work_dev, void* cuda_stream);

/* One Adam step (Kingma & Ba) on n parameters, step number t >= 1:
 * m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
 * s <- s - lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps).  All arrays double,
 * device memory, caller-owned; m and v start at zero. */
llg_status llg_adam_step(double* s_dev, const double* grad_dev, double* m_dev, double* v_dev, int n, long long t,
                         double lr, double b1, double b2, double eps, void* cuda_stream);

/* Host-only: the checkpoint action list the library executes.  Writes up to
 * max_actions triples (op, a, b) to `actions` (forward actions first, then
 * reverse), sets *n_forward to the number of forward actions and returns the
 * total count (or -1 on bad arguments).  ops: 0 SNAP (n, slot), 1 ADVANCE
 * (n0, n1), 2 RESTORE (slot, n), 3 RECORD (n0, n1), 4 REVERSE (n1, n0).
 * Every list works on one working state: RESTORE loads it from a slot,
 * ADVANCE moves it, SNAP stores it, RECORD records its next steps' stage
 * data; the objective accumulates only in the forward actions. */
long long llg_schedule(long long nsteps, int ckpt, int seg_len, long long* actions,
                       long long max_actions, long long* n_forward);

/* Host-only: padded in-plane FFT extents the library uses for a grid (Px,
 * Py); the padded z extent of a 3D grid is the power of two >= 2 nz. */
int llg_padded_extents(int nx, int ny, int* Px, int* Py);

int llg_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LLG_H */
