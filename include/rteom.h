/*
 * rteom.h -- C ABI of the B300 RT-EOM-CCSD core-hole propagation library
 * (librteom.so).
 *
 * The library propagates the coupled-cluster singles and doubles amplitudes
 * of one core-ionised (N-1)-electron reference in real time and accumulates
 * the cumulant C(t) of the core-hole Green's function (Pathak et al.,
 * "Real-time Equation-of-Motion Coupled-Cluster Cumulant Green's Function
 * Method", Section 2.1 Eqs. 1-8 and Section 3 Eq. 9).  All arithmetic runs in
 * the library's CUDA kernels on one GPU; the host only copies inputs in and
 * results out.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - nocc (O) occupied and nvir (V) virtual spatial orbitals of the
 *    N-electron closed-shell system, nb = O + V; O counts the core orbital.
 *  - The ionised electron is the beta copy of spatial orbital core_index
 *    (0 <= core_index < O).  Spin spaces of the (N-1) reference:
 *      alpha occupied = spatial 0..O-1                         (oA = O)
 *      beta  occupied = spatial 0..O-1 without core_index       (oB = O-1)
 *      alpha virtual  = spatial O..nb-1                        (vA = V)
 *      beta  virtual  = [core_index, O..nb-1] (core first)     (vB = V+1)
 *  - "Amplitude vector": the unique spin blocks of Section 3.1.1, complex128
 *    stored as interleaved (re, im) doubles, concatenated in this order and
 *    each row-major:
 *      t1a[oA][vA], t1b[oB][vB], t2aa[oA][oA][vA][vA], t2ab[oA][oB][vA][vB],
 *      t2bb[oB][oB][vB][vB];
 *    t2aa and t2bb are antisymmetric in (i,j) and in (a,b).  Its length in
 *    doubles is rteom_state_size().
 *  - Every function returns RTEOM_OK (0) or a negative RTEOM_ERR_* code and
 *    never aborts the process; rteom_last_error() gives a message.  After
 *    RTEOM_ERR_CUDA the context must be destroyed.
 *  - A context is not thread-safe; distinct contexts are independent.  All
 *    device work of a context runs on the stream given at creation.
 *  - Host pointers are read or written only during the call; the caller
 *    keeps ownership of every buffer it passes.
 */
#ifndef RTEOM_H
#define RTEOM_H

#ifdef __cplusplus
extern "C" {
#endif

#define RTEOM_OK                 0
#define RTEOM_ERR_ARG           -1   /* bad size, index, pointer or value          */
#define RTEOM_ERR_OOM           -2   /* device memory exhausted                     */
#define RTEOM_ERR_CUDA          -3   /* CUDA runtime error (context unusable)       */
#define RTEOM_ERR_NOT_CONVERGED -4   /* micro-iteration cap reached (Eq. 9)         */
#define RTEOM_ERR_NONFINITE     -5   /* NaN/Inf in an input or in the amplitudes    */
#define RTEOM_ERR_STATE         -6   /* call not valid in the context's state       */

/* precision forms */
#define RTEOM_FP64        0   /* every contraction and update in FP64           */
#define RTEOM_SPLIT_BF16  1   /* contractions of at least 5e7 FLOP (and smaller
                                 ones the autotuner finds faster there) on the
                                 BF16 tensor cores as three 8-bit digit planes
                                 per operand with per-row power-of-two scales
                                 (x carried to about 2^-24 of its row scale):
                                 the leading digit-pair product summed exactly
                                 in FP32 over chunks of 512 of K, the 5 other
                                 leading pairs (planes pre-scaled by their
                                 digit weights) in one FP32 accumulator
                                 beside it, chunks added as compensated
                                 pairs; complex x complex products as three
                                 real ones; every other step FP64 */
#define RTEOM_SPLIT_TF32  2   /* contractions of at least 5e7 FLOP (and smaller
                                 ones the autotuner finds faster there) on the
                                 tensor cores as split-TF32 products (x = hi +
                                 lo, hi*hi + hi*lo + lo*hi) with FP32
                                 accumulation over slices of at most 512 of K,
                                 slices summed as compensated FP32 pairs;
                                 complex x complex products as three real ones;
                                 every other step (small contractions,
                                 Adams-Moulton update, cumulant, phases) FP64 */
#define RTEOM_FP64_OZAKI  3   /* FP64-accurate contractions on the BF16 tensor
                                 cores (no counterpart in the paper): operands
                                 sliced into seven 8-bit digit planes with
                                 per-row power-of-two scales (Ozaki et al.,
                                 Numer. Algorithms 59, 2012), the 28 leading
                                 digit-pair products summed exactly in FP32 over
                                 chunks of 128 of K and accumulated as
                                 compensated pairs (about 2^-48 relative to the
                                 row scales); contractions below 5e7 FLOP and
                                 every other step as in RTEOM_FP64 */
#define RTEOM_SPLIT_FP16  4   /* contractions of at least 5e7 FLOP (and smaller
                                 ones the autotuner finds faster there) on the
                                 16-bit tensor cores as split-FP16 products:
                                 each operand row scaled by a power of two
                                 into FP16's range, x = hi + lo in two FP16
                                 planes (11 significant bits each, as split
                                 TF32), hi*hi + hi*lo + lo*hi in one FP32
                                 accumulator over chunks of 512 of K, chunks
                                 added as compensated pairs; twice the TF32
                                 tensor rate; complex x complex products as
                                 three real ones; every other step FP64 */

/* flags for rteom_create */
#define RTEOM_FLAG_CUMULANT_NO_FOV 1  /* cumulant integrand without sum f_ia t_i^a,
                                         i.e. Eq. 6 as printed; default keeps it
                                         (the definition in Eq. 5)              */
#define RTEOM_FLAG_LADDER_CHOLESKY 2  /* Cholesky mode: keep no (ov|vv) or
                                         (vv|vv) block on the device; the
                                         particle-particle ladder (Section
                                         3.1.1) and the other terms with three
                                         or four virtual indices are formed
                                         from the Cholesky vectors at every
                                         residual, in chunks of a (and of m).
                                         rteom_create takes this mode by itself
                                         when the resident blocks do not fit
                                         the free device memory; nchol == 0
                                         keeps the resident mode             */
#define RTEOM_FLAG_ANDERSON        4  /* Anderson-accelerated micro-iterations
                                         (no counterpart in the paper, which
                                         names faster solvers of the implicit
                                         step as future work, Section 3):
                                         x_{k+1} = g_k - sum_j gamma_j dG_j
                                         over the last 3 differences of
                                         g = G(x) and f = g - x, gamma the
                                         least-squares fit of f (Walker and
                                         Ni, SIAM J. Numer. Anal. 49, 2011).
                                         Same stopping rule |g_k - x_k| < tol
                                         and the same accepted value g_k, so
                                         the step converges to the same
                                         implicit solution in fewer residuals
                                         at tight tol; 9 extra amplitude-sized
                                         device vectors                       */
#define RTEOM_FLAG_GROUPED         8  /* grouped ladder, for running many
                                         propagations in lock step
                                         (rteom_propagate_group): every
                                         residual forms tau and packs the
                                         operands of its three ladder GEMMs
                                         (Section 3.1, sum_cd v_abcd tau_ij^cd)
                                         first, the GEMMs run as one grouped
                                         persistent launch (with those of the
                                         other contexts of a group), then the
                                         rest of the residual adds their
                                         results.  Each ladder GEMM takes one K
                                         range per output tile, so a context's
                                         results are the same bits alone and in
                                         any group.  Needs RTEOM_FP64_OZAKI,
                                         RTEOM_SPLIT_BF16 or RTEOM_SPLIT_FP16
                                         and the resident ladder blocks (not
                                         with RTEOM_FLAG_LADDER_CHOLESKY or
                                         RTEOM_FLAG_ANDERSON; RTEOM_ERR_OOM
                                         when they do not fit); no timing
                                         modes.  rteom_propagate and the
                                         server run such a context as a group
                                         of one                               */

typedef struct rteom_ctx rteom_ctx;

/*
 * rteom_create -- set up one core-hole propagation (Section 3, workflow
 * steps "read the N-electron orbitals into the (N-1) space and build the
 * (N-1) Fock matrix"; f_pq = eps_p delta_pq - <pc||qc>, Section 2.1).
 *
 *  out        receives the new context (set to NULL on failure)
 *  nocc,nvir  O >= 1, V >= 1;  nchol >= 0 Cholesky vectors
 *  eps        host [nb] N-electron Hartree-Fock orbital energies (Ha)
 *  L          host [nchol][nb][nb] real Cholesky vectors of the two-electron
 *             integrals, (pq|rs) = sum_Q L[Q][p][q] L[Q][r][s]; must satisfy
 *             L[Q][p][q] == L[Q][q][p]; may be NULL when nchol == 0
 *  t1_gs      host [O][V] closed-shell ground-state T1, or NULL (zero)
 *  t2_gs      host [O][O][V][V] closed-shell (alpha-beta) ground-state T2, or
 *             NULL; t1_gs/t2_gs only enter E_N^corr of Eq. 3:
 *             E = sum_ijab [2(ia|jb) - (ib|ja)] (t_ij^ab + t_i^a t_j^b)
 *  core_index spatial index c of the ionised orbital, 0 <= c < O
 *  precision  RTEOM_FP64, RTEOM_SPLIT_BF16, RTEOM_SPLIT_TF32,
 *             RTEOM_FP64_OZAKI or RTEOM_SPLIT_FP16
 *  flags      RTEOM_FLAG_* bits
 *  cuda_stream cudaStream_t to run on, or NULL for a non-blocking stream
 *             created and owned by the context
 *
 * The inputs are copied to device memory owned by the context (cudaMalloc);
 * the amplitudes start at T(0) = 0 and C(0) = 0 (Section 3).  Errors:
 * RTEOM_ERR_ARG (sizes, indices, NULL eps), RTEOM_ERR_NONFINITE (NaN/Inf in
 * an input), RTEOM_ERR_OOM, RTEOM_ERR_CUDA.  Fault injection for tests: with
 * the environment variable RTEOM_INJECT_DEVICE_LIMIT=<bytes> set when the
 * context is created, its device allocations past that total fail with
 * RTEOM_ERR_OOM on the host (no device call is made for them).
 */
int rteom_create(rteom_ctx** out, int nocc, int nvir, int nchol,
                 const double* eps, const double* L,
                 const double* t1_gs, const double* t2_gs,
                 int core_index, int precision, int flags, void* cuda_stream);

/*
 * rteom_propagate -- advance the amplitudes nsteps time steps of length dt
 * with the first-order Adams-Moulton rule (Eq. 9), each solved by fixed-point
 * micro-iterations (Anderson-accelerated with RTEOM_FLAG_ANDERSON) from the
 * predictor t^(0) = t_n, stopping when the largest
 * |t^(k+1) - t^(k)| over all blocks is below tol, and accumulate the cumulant
 * C_{n+1} = C_n + (i dt/2)(E_n + E_{n+1}) with E = <Phi|(H_N e^T)_C|Phi>
 * (Eqs. 5-6).
 *
 *  nsteps     >= 0;  dt > 0 (au) and equal in every call of a context (the
 *             first propagate call fixes it; a state restored with
 *             rteom_set_state carries no dt, so the caller keeps it equal)
 *  tol        > 0 micro-iteration cutoff (the paper uses 1e-4)
 *  max_micro  >= 1 cap on micro-iterations per step
 *  C_out      host [nsteps+1] complex (2*(nsteps+1) doubles) or NULL:
 *             C at the start of this call and after each of its steps.
 *
 * Returns RTEOM_ERR_NOT_CONVERGED if a step hits max_micro (the context keeps
 * the last completed step), RTEOM_ERR_NONFINITE if the amplitudes become
 * non-finite, RTEOM_ERR_ARG for bad arguments.
 */
int rteom_propagate(rteom_ctx* ctx, int nsteps, double dt, double tol, int max_micro,
                    double* C_out);

/*
 * rteom_propagate_group -- rteom_propagate for n contexts at once, in lock
 * step (no counterpart in the paper, whose core-hole propagations are
 * independent and run side by side, Section 3).  In every round each member
 * with steps left evaluates one residual (R(t_n) of its next step or
 * R(t^(k)) of its next micro-iteration) and its Adams-Moulton update; the
 * ladder GEMMs of all members of the round run as grouped persistent
 * tensor-core launches (one per output-tile width, up to 16 GEMMs each) on
 * the first member's stream, between the members' captured graphs of the
 * residual's two parts on their own streams.  Members may differ in
 * (O, V, Nchol); they advance by the same stopping rule as rteom_propagate,
 * each with its own number of micro-iterations, and each result equals that
 * of rteom_propagate on the member alone, bit for bit.
 *
 *  ctxs       n distinct contexts created with RTEOM_FLAG_GROUPED and one
 *             precision form; 1 <= n <= 1024; their streams may differ
 *  nsteps, dt, tol, max_micro   as for rteom_propagate, for every member
 *  C_out      NULL, or n pointers (each NULL or host [nsteps+1] complex):
 *             member i's C at the start of the call and after each step
 *
 * Errors: RTEOM_ERR_ARG (bad arguments, a member without the flag, mixed
 * forms, a repeated member; reported on that member); the first member
 * error of a round (RTEOM_ERR_NOT_CONVERGED, RTEOM_ERR_NONFINITE,
 * RTEOM_ERR_CUDA) stops the call and is reported on that member; the other
 * members keep their last completed step.
 */
int rteom_propagate_group(rteom_ctx* const* ctxs, int n, int nsteps, double dt, double tol,
                          int max_micro, double* const* C_out);

/*
 * rteom_spectrum -- core spectral function A(w) = -(1/pi) Im G^R(w)
 * (Section 2.1) of everything propagated so far: with
 * G_n = -i exp(-i (eps_c + E_corr) tau_n) exp(C_n) (Eq. 4), tau_n = n dt,
 *   A(w_m) = -(1/pi) Im sum_{n=0}^{M} w_n dt G_n exp(i w_m tau_n - eta tau_n),
 * trapezoid weights w_0 = w_M = 1/2, others 1.
 *
 *  omega  host [nomega] frequencies (Ha);  eta >= 0 damping (Ha)
 *  A_out  host [nomega]
 * Errors: RTEOM_ERR_STATE if no step has been propagated, RTEOM_ERR_ARG.
 */
int rteom_spectrum(rteom_ctx* ctx, const double* omega, int nomega, double eta,
                   double* A_out);

/*
 * rteom_get_info -- scalars of the propagation.  Any output pointer may be
 * NULL.  eps_core = eps[core_index]; e_corr = E_N^corr (Eq. 3);
 * steps_done and micro_total count the steps and micro-iterations so far.
 */
int rteom_get_info(const rteom_ctx* ctx, double* eps_core, double* e_corr,
                   long long* steps_done, long long* micro_total);

/* rteom_state_size -- length in doubles of the amplitude vector (see top). */
long long rteom_state_size(const rteom_ctx* ctx);

/*
 * rteom_get_cumulant -- copy C_0..C_{count-1} (count <= steps_done + 1) and
 * the matching cumulant integrands E_n into host arrays of 2*count doubles
 * each (interleaved complex); either pointer may be NULL.
 */
int rteom_get_cumulant(const rteom_ctx* ctx, long long count, double* C_out, double* E_out);

/*
 * rteom_get_state / rteom_set_state -- checkpoint and restart (Section 3.1.1,
 * "Restarting the time propagation ... requires the T amplitudes").  The
 * state is the amplitude vector t_n plus the step count; the cumulant
 * history (C_0..C_n, E_0..E_n) travels with it so the spectrum stays
 * complete.  t_out/t_in: host amplitude vector (rteom_state_size doubles).
 * hist: host [2*(steps+1)] C followed by [2*(steps+1)] E, or NULL to skip
 * (get) / to restart the history at this state with C = 0 (set).
 * set_state also lets tests start from a chosen T(0).  Padding-free; the
 * entries of t2aa/t2bb must be antisymmetric (not checked beyond finiteness).
 */
int rteom_get_state(const rteom_ctx* ctx, double* t_out, long long* steps, double* hist);
int rteom_set_state(rteom_ctx* ctx, const double* t_in, long long steps, const double* hist);

/*
 * rteom_plan_bytes -- device memory of a context of this shape and precision,
 * planned on the host from the same dry run of the residual that sizes
 * rteom_create's scratch arena (no device calls; usable without a GPU).  The
 * paper has no counterpart (capacity planning of contexts before creating them).
 *  bytes  host double[3]: [0] peak during set-up and the first residual with
 *         every constant tensor-core pack cached (what rteom_create takes
 *         when memory allows), [1] the same with no pack cached (the least
 *         it works with), [2] held after set-up with every pack cached
 *  flags  RTEOM_FLAG_LADDER_CHOLESKY plans the Cholesky mode; without it
 *         the plan has resident (ov|vv)/(vv|vv) blocks; RTEOM_FLAG_ANDERSON
 *         adds the buffers of the accelerated micro-iteration
 * Returns RTEOM_OK, or RTEOM_ERR_ARG for a bad shape, precision or flag.
 */
int rteom_plan_bytes(int nocc, int nvir, int nchol, int precision, int flags, double* bytes);

/*
 * rteom_debug_residual -- test entry point: evaluate the full projections
 * R_mu = <Phi_mu|(H_N e^{T1+T2})_C|Phi> (Eqs. 7-8) and the cumulant
 * integrand E (Eq. 5) for given amplitudes, without changing the state.
 * t_in, R_out: host amplitude vectors; E_out: host [2] (may be NULL).
 */
int rteom_debug_residual(rteom_ctx* ctx, const double* t_in, double* R_out, double* E_out);

/*
 * rteom_debug_residual_sparse -- test entry point for problems whose
 * amplitude vector is too large to pass through the host: the projections
 * R_mu of Eqs. 7-8 at chosen entries, for amplitudes that are zero except
 * at chosen entries (the context's state is not changed).
 *  t_index, t_val, nt  host: nt flat complex indices into the amplitude
 *                      vector (0 <= k < rteom_state_size/2) and their values
 *                      (2*nt doubles, interleaved); every other amplitude is
 *                      zero.  Entries of t2aa/t2bb must come with their
 *                      antisymmetric partners (not checked).  Repeated
 *                      indices: one of the values is kept.
 *  r_index, nr, R_out  host: nr flat indices and the residual there
 *                      (2*nr doubles)
 * A residual depends on the orbitals its amplitudes touch: every summed
 * index of a CCSD term sits on an amplitude.  So for amplitudes supported on
 * a few orbitals the entries returned equal the residual of the problem cut
 * down to those orbitals and the free ones, which tests compare with the
 * oracle at full problem sizes.  Errors: RTEOM_ERR_ARG (an index outside the
 * vector, missing arrays), RTEOM_ERR_NONFINITE, RTEOM_ERR_OOM,
 * RTEOM_ERR_CUDA.
 */
int rteom_debug_residual_sparse(rteom_ctx* ctx, const long long* t_index, const double* t_val,
                                long long nt, const long long* r_index, long long nr,
                                double* R_out);

/*
 * rteom_set_timing / rteom_get_timing -- per-kernel-class device timing with
 * CUDA events on the context's stream (0 = off, the default).  Classes:
 * 0 ladder contraction, 1 other contractions, 2 tensor permutes (and
 * tensor-core operand packing), 3 elementwise/update/energy.  get_timing
 * fills ms[4] (total milliseconds), launches[4] and flops[4] (FP64-equivalent
 * algorithmic FLOPs of the launches: 2, 4 or 8 per real, mixed or complex
 * multiply-add of each contraction as posed on the slot spaces; the split
 * and emulated forms execute that many times the products per multiply-add
 * on the tensor cores), bytes[4] (algorithmic DRAM bytes: operands read once,
 * outputs or split-K slabs written); any pointer may be NULL.  reset != 0
 * zeroes the counters after reading.  Modes: on = 1 puts event nodes inside
 * the captured residual graphs around the ladder launches only, so ms[] of
 * the other classes counts only eagerly launched work (set-up,
 * rteom_debug_residual); launches[] and flops[] count every launch.  on = 3
 * puts event nodes around every contraction launch (classes 0 and 1).
 * on = 2 runs the residuals of rteom_propagate eagerly (no graphs, the same
 * kernels) with an event pair around every launch, so every class is timed;
 * with the environment variable RTEOM_TRACE=<file> each timed launch also
 * appends one JSON line (class, contraction, FLOPs, ms) to that file.
 * Errors: RTEOM_ERR_ARG for a mode outside 0..3.
 */
int rteom_set_timing(rteom_ctx* ctx, int on);
int rteom_get_timing(rteom_ctx* ctx, double* ms, long long* launches, double* flops,
                     double* bytes, int reset);

/* rteom_kernel_launches -- number of kernels this context has launched. */
long long rteom_kernel_launches(const rteom_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Continuous-batching server.  Core holes are independent (Section 3: the
 * core-hole calculations "are unique and can run simultaneously"), so one
 * GPU propagates many of them at once.  A scheduler thread owned by the
 * server admits queued requests first come, first served, while a slot is
 * free and the request's estimated device memory fits the budget; each
 * admitted request gets its own context and stream and is advanced by
 * non-blocking polls, so the work of different requests overlaps on the
 * device and late arrivals join as soon as slots and memory free up.  Results
 * are bitwise identical to a lone rteom_propagate of the same request.  A
 * failing request (bad input, NOT_CONVERGED, ...) is isolated.
 * The server functions are thread-safe.
 * ------------------------------------------------------------------------- */
#define RTEOM_REQ_QUEUED    0
#define RTEOM_REQ_RUNNING   1
#define RTEOM_REQ_DONE      2
#define RTEOM_REQ_FAILED    3
#define RTEOM_REQ_CANCELLED 4

typedef struct rteom_server rteom_server;

/*
 * rteom_server_create -- start a server on the current CUDA device.
 *  mem_budget_bytes  device memory the running requests may hold (0: 80 % of
 *                    the free memory at creation)
 *  max_active        slots: requests running at once (>= 1)
 *  precision         one of the RTEOM_* precision forms, for every request
 */
int rteom_server_create(rteom_server** out, double mem_budget_bytes, int max_active,
                        int precision);

/*
 * rteom_server_submit -- queue one propagation: the arguments of
 * rteom_create and rteom_propagate (host arrays are copied; the caller may
 * free them on return).  *request_id receives the request's id.
 * Running requests with RTEOM_FLAG_GROUPED (digit-plane server forms) step
 * together: in every pass of the scheduler, those whose last micro-iteration
 * has finished evaluate their next residual with all their ladder GEMMs in
 * grouped launches (see rteom_propagate_group); the others keep running and
 * join a later pass.  Results are the same bits as the request alone.
 */
int rteom_server_submit(rteom_server* s, int nocc, int nvir, int nchol, const double* eps,
                        const double* L, const double* t1_gs, const double* t2_gs,
                        int core_index, int flags, int nsteps, double dt, double tol,
                        int max_micro, long long* request_id);

/*
 * rteom_server_submit_sweep -- queue one propagation per core hole c in
 * cores[] of the same molecule (Section 3: the core-hole calculations of one
 * system are independent and can run at the same time).  The host inputs
 * are copied once and shared by the requests until each has built its
 * context; every request builds its own (N-1) Fock matrix and integral
 * blocks on the device, since both depend on c.
 *  cores        host int[ncores], each 0 <= c < nocc; ncores >= 1
 *  request_ids  host long long[ncores]: the ids, in the order of cores
 * The other arguments are those of rteom_server_submit.  A bad argument
 * returns RTEOM_ERR_ARG and queues nothing.
 */
int rteom_server_submit_sweep(rteom_server* s, int nocc, int nvir, int nchol, const double* eps,
                              const double* L, const double* t1_gs, const double* t2_gs,
                              const int* cores, int ncores, int flags, int nsteps, double dt,
                              double tol, int max_micro, long long* request_ids);

/*
 * rteom_server_poll -- state of a request.  status: RTEOM_REQ_*; error: the
 * RTEOM_ERR_* code of a failed request; C_out (host, 2*(nsteps+1) doubles or
 * NULL) receives C_0..C_nsteps once the request is DONE; times (host [3] or
 * NULL): submit, admit and completion times in seconds since the server
 * started (-1 when not reached).  Unknown id: RTEOM_ERR_ARG.
 */
int rteom_server_poll(rteom_server* s, long long id, int* status, int* error, double* C_out,
                      double* times);

/* rteom_server_wait -- block until the request is done, failed or cancelled
 * (timeout_s <= 0: no limit); RTEOM_ERR_STATE on timeout. */
int rteom_server_wait(rteom_server* s, long long id, double timeout_s);

/* rteom_server_cancel -- cancel a queued or running request. */
int rteom_server_cancel(rteom_server* s, long long id);

/* rteom_server_stats -- queued/running/done/failed counts, device bytes held
 * by running requests, and time steps completed by finished requests; any
 * pointer may be NULL. */
int rteom_server_stats(rteom_server* s, long long* queued, long long* running, long long* done,
                       long long* failed, double* mem_in_use, double* steps_done);

/* rteom_server_estimate_bytes -- the admission estimate of a request's peak
 * device memory for this shape and precision. */
double rteom_server_estimate_bytes(int nocc, int nvir, int nchol, int precision);

/* rteom_server_destroy -- cancel what is left, stop the thread, free all. */
void rteom_server_destroy(rteom_server* s);

/*
 * rteom_ecorr_noalloc -- the closed-shell correlation energy E_N^corr that
 * rteom_create computes (sum_ijab [2(ia|jb) - (ib|ja)] (t_ij^ab + t_i^a t_j^b),
 * (pq|rs) = sum_Q L[Q][p][q] L[Q][r][s]), for callers that must not allocate
 * device memory.  The paper has no counterpart: this entry point exists for
 * programs whose device memory is owned entirely by their own pool or
 * framework allocator, or that run where a cudaMalloc/cudaFree (which may
 * synchronise the device) is not allowed.  It allocates nothing: no
 * cudaMalloc, cudaFree or allocating library call.
 *
 *  nocc, nvir, nchol  as for rteom_create; nocc*nocc <= 4096 (nocc <= 64)
 *  L, t1_gs, t2_gs    DEVICE pointers, layouts as for rteom_create (t1_gs,
 *                     t2_gs may be NULL: zero); L may be NULL if nchol == 0
 *  e_corr             DEVICE pointer to one double, written asynchronously
 *  cuda_stream        cudaStream_t, or NULL for the legacy default stream
 *  err, err_len       optional host buffer for an error message (may be NULL)
 *
 * Scratch: one partial sum per occupied pair lives in a static device array
 * of 4096 doubles (32 KiB) that every GPU loading the library keeps until the
 * process exits.  The first call in each CUDA context (the first call on a
 * device, and the first again after a cudaDeviceReset, which reloads the
 * library's device code at a new address) looks up that array's device
 * address with cudaGetSymbolAddress, with the caller's device current, and
 * caches it under the context's id; make that first call before any stream
 * capture.  All calls share the array and each overwrites the partials it
 * reads, so calls whose kernels overlap on the GPU (other streams, other host
 * threads) race and must be serialised.
 * Cost: 2 O^2 V^2 Nchol FP64 FMAs (the integrals are formed from L for every
 * (i,j,a,b)), meant for small ground-state problems.
 * Errors: RTEOM_ERR_ARG (sizes, including nocc*nocc > 4096, or NULL
 * pointers; checked before any launch), RTEOM_ERR_CUDA.
 */
int rteom_ecorr_noalloc(int nocc, int nvir, int nchol, const double* L,
                        const double* t1_gs, const double* t2_gs, double* e_corr,
                        void* cuda_stream, char* err, int err_len);

/* rteom_destroy -- free every device and host resource of the context. */
void rteom_destroy(rteom_ctx* ctx);

/*
 * rteom_last_error -- message of the last failed call on ctx, or of the last
 * failed rteom_create on this thread when ctx is NULL.  Valid until the next
 * call on the same context/thread.
 */
const char* rteom_last_error(const rteom_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* RTEOM_H */
