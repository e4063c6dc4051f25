/*
 * dirac.h -- C ABI of libdirac_gb300.so: the Crank-Nicolson time step of the 3D time-dependent
 * Dirac equation in a dual-kinetic-balance B-spline x spherical-spinor basis, on one GB300
 * (sm_103a).  Method: arXiv 2512.21697 ("GaDE"), Sec. 2 (theory) and Sec. 3 (time loop).
 *
 * Conventions shared by every call
 *  - Atomic units.  Every call returns a dirac_status; on failure dirac_last_error() returns a
 *    thread-local message.  Parameters are validated before anything is allocated.  No C++
 *    exception crosses this boundary.
 *  - Device buffers are plain device pointers owned by the caller (e.g. torch tensors'
 *    data_ptr()); the library never frees them.  Opaque handles are owned by the library and
 *    released with the matching *_free call.
 *  - All device work is ordered on the CUDA stream given to dirac_operator_setup.  Calls that
 *    return host-visible numbers synchronise that stream before returning.
 *  - State vectors are complex128 (interleaved re, im doubles), "library order": channel-major
 *    (channels as listed by dirac_basis_channels), then radial slot r = 0 .. N, then DKB type
 *    (0 = large: P = u, Q = (u' + kappa u / r)/2c; 1 = small: P = (u' - kappa u / r)/2c, Q = u;
 *    Eq. dualkinetic), where slot r carries B-spline B_{r+1} of the knot vector B_0 .. B_{N+3}.
 *    Length n = n_channels * 2 (N + 1).  The zero boundary condition at r = 0 (Sec. 2.2) leaves
 *    slot 0 type 0 used only for kappa = -1 and slot 0 type 1 only for kappa = +1; those unused
 *    entries must be zero on input and stay zero (the operators act on them as the identity).
 */
#ifndef DIRAC_GB300_H
#define DIRAC_GB300_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DIRAC_OK = 0,
    DIRAC_E_ARG = 1,        /* invalid argument (nothing was allocated or changed)           */
    DIRAC_E_NOMEM = 2,      /* host or device allocation failed                              */
    DIRAC_E_CUDA = 3,       /* a CUDA runtime call failed (message names it)                 */
    DIRAC_E_NOCONV = 4,     /* BiCGSTAB hit max_iter before tol                              */
    DIRAC_E_BREAKDOWN = 5,  /* BiCGSTAB breakdown persisted after one restart                */
    DIRAC_E_NUMERIC = 6,    /* non-finite residual                                           */
    DIRAC_E_STATE = 7       /* handle in the wrong state (e.g. no GPU, freed basis)          */
} dirac_status;

typedef struct dirac_basis dirac_basis; /* host-side basis and operator data                  */
typedef struct dirac_op dirac_op;       /* device operator, factors, workspaces               */
typedef struct dirac_guess dirac_guess; /* learned initial-guess network and its training state */

/* Radial and angular discretisation (Sec. 2.2).  n_splines = N B-splines kept for every kappa
 * (B_2 .. B_{N+1}); order = B-spline order k; grid 0 = linear breakpoints on [0, R]; grid 1 =
 * n_lin linear intervals up to r_lin then geometrically growing intervals up to R (the growth
 * factor is fixed by the interval count N + 5 - k); kappa_max bounds |kappa|; two_mu_max bounds
 * |2 mu| (<= 0: every mu); l_max truncates the multipole (plane-wave) expansion of the pulse
 * (Eq. bdpA); quad_pts = Gauss-Legendre points per knot interval. */
typedef struct {
    double Z, c, R;
    int n_splines, order, grid;
    double r_lin;
    int n_lin, kappa_max, two_mu_max, l_max, quad_pts;
} dirac_basis_params;

/* sin^2 pulse, Eq. (ndpPot): A_x = (E0/omega) sin^2(pi (t-z/c)/T) sin(omega (t-z/c)),
 * T = n_cycles 2 pi / omega, polarised along x, travelling along z, on for 0 <= t <= T.
 * t0 shifts the pulse start (field at time t uses t - t0). */
typedef struct {
    double E0, omega, n_cycles, t0;
} dirac_pulse;

/* Time stepping (Eq. solPsi) and its BiCGSTAB solve.
 * dt: step; tol: relative residual ||b - A_+ x|| / ||b||; max_iter: BiCGSTAB iteration cap per
 * step (per inner solve in mixed precision); precision: 0 = FP64 throughout, 1 = complex64
 * BiCGSTAB inside FP64 iterative refinement, 2 = as 1 with the double-precision-accurate parts
 * (coupling assembly, A_- psi, refinement residuals) in double-float arithmetic (FP32 hi/lo pairs,
 * error-free transforms; about 2^-44 relative per operation); tol_inner: inner relative
 * tolerance (precision >= 1); max_outer: refinement cap (precision >= 1); guess: 0 = psi_n, 1 = quadratic extrapolation,
 * 2 = learned (dirac_op_set_guess; falls back to 1 without a network or history)
 * 3 psi_n - 3 psi_{n-1} + psi_{n-2}; time_eval: 0 = H at t + dt/2 (midpoint rule of Sec. 2.4),
 * 1 = H at t + dt (Eq. solPsi as printed); precond: 0 = none, 1 = LU of M = S + i dt/2 H0
 * (Eq. matrixM). */
typedef struct {
    double dt, tol, tol_inner;
    int max_iter, precision, max_outer, guess, time_eval, precond;
} dirac_solver_opts;

/* Build the basis, the kappa-polynomial radial matrices h_n, s_n (Eq. fullH and Sec. 2.3), the
 * projected pulse matrices g^n_{alpha,l} (Eq. fullH), the angular coefficients H^theta_l
 * (Eq. Htheta via Eq. HthetaExpand and Eq. GauntCoef) and the channel-pair list.  Host only.
 * psi0_host (nullable, n complex128 in library order): receives the 1s1/2, mu = +1/2 state,
 * the lowest kappa = -1 solution of H0 v = E S v above -c^2 (Sec. 2.3), v^T S v = 1, largest
 * component positive.  e0 (nullable) receives its energy. */
dirac_status dirac_basis_build(const dirac_basis_params* params, dirac_basis** out,
                               double* psi0_host, double* e0);
void dirac_basis_free(dirac_basis* basis);
int64_t dirac_basis_dim(const dirac_basis* basis);          /* n, or -1 for NULL            */
int dirac_basis_nchannels(const dirac_basis* basis);
/* channel labels in library order: kappa[i], two_mu[i] (host arrays of n_channels ints) */
dirac_status dirac_basis_channels(const dirac_basis* basis, int* kappa, int* two_mu);
/* number of coupled unordered channel pairs (a < b) */
int64_t dirac_basis_npairs(const dirac_basis* basis);
/* number of (pair, multipole l) terms of the coupling, Sec. 2.2 Eq. fullH: the multipoles with a
 * nonzero angular coefficient (Eq. Htheta) summed over the pairs; -1 for a NULL basis */
int64_t dirac_basis_nterms(const dirac_basis* basis);
/* Host copies of setup data for parity checks.  Radial blocks of one kappa as dense
 * (2(N+1))^2 row-major matrices in library order (slot-major, type-minor). */
dirac_status dirac_basis_radial(const dirac_basis* basis, int kappa, double* S, double* H0);
/* Coupling block X_ab(t) of H_ab = i X_ab (Eq. fullH) for channels a != b (library indices),
 * dense (2(N+1))^2 row-major in library order, pulse and time t given.  Host only. */
dirac_status dirac_basis_coupling(const dirac_basis* basis, const dirac_pulse* pulse, int a, int b,
                                  double t, double* X);
/* 4 pi Y_l0(z) <X_{k1 m1}| sigma_x Y_l0 |X_{k2 m2}> (the Eq. Htheta coefficient with the
 * bra's kappa written out), two_mu = 2 mu. */
double dirac_angular(int kappa1, int two_mu1, int kappa2, int two_mu2, int l);

/* Upload the operator for one pulse and solver setting: radial blocks, pulse matrices, pair
 * coefficients and the block-banded LU factors of M = S + i dt/2 H0, and allocate every device
 * workspace (coupling values, Krylov vectors).  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream).  Device memory is reported by dirac_op_device_bytes. */
dirac_status dirac_operator_setup(const dirac_basis* basis, const dirac_pulse* pulse,
                                  const dirac_solver_opts* opts, void* cuda_stream, dirac_op** out);
void dirac_op_free(dirac_op* op);
int64_t dirac_op_device_bytes(const dirac_op* op);

/* y = A_sign(t) x, A_+- = S +- i dt/2 H(t) (Eq. solPsi), H evaluated at time t.  Assembles the
 * coupling values for t first.  x_dev, y_dev: device complex128[n], must not alias. */
dirac_status dirac_apply(dirac_op* op, int sign, double t, const void* x_dev, void* y_dev);
/* z = M^-1 r with M = S + i dt/2 H0 (Eq. matrixM).  r_dev, z_dev: device complex128[n]. */
dirac_status dirac_precond_apply(dirac_op* op, const void* r_dev, void* z_dev);

/* Advance psi by n_steps Crank-Nicolson steps starting at t_start (step s covers
 * [t_start + s dt, t_start + (s+1) dt]): psi <- A_+^{-1} A_- psi, each solve by BiCGSTAB
 * (precision 0) or mixed-precision refinement (precision 1) to opts.tol.
 * psi_dev: device complex128[n], in/out.  hist_dev: nullable device complex128[2n] holding
 * psi_{n-1}, psi_{n-2} for the extrapolated guess; n_hist (nullable, in/out) says how many of
 * them are valid (0..2) -- with NULL history the guess restarts from psi_n.
 * iters_out / resid_out: nullable host arrays of n_steps receiving BiCGSTAB iterations (total
 * inner iterations in precision 1) and the final relative residual per step.
 * Returns DIRAC_E_NOCONV / DIRAC_E_BREAKDOWN / DIRAC_E_NUMERIC if a step fails (psi then holds
 * the last iterate of that step). */
dirac_status dirac_step(dirac_op* op, void* psi_dev, void* hist_dev, int* n_hist, int n_steps,
                        double t_start, int* iters_out, double* resid_out);

/* dirac_step as one captured CUDA graph: the time loop, the solve restarts and the BiCGSTAB
 * iterations are conditional WHILE nodes whose conditions the device sets from the solver state,
 * so n_steps run with no host round trip (same arithmetic, kernel sequence and results as
 * dirac_step).  hist_dev (device complex128[2n], [3n] with the learned guess) is required; n_hist
 * as in dirac_step.  The graph
 * is captured on the first call and re-captured when psi_dev or hist_dev changes or n_steps grows
 * beyond the previous capacity (at least 256).  Same outputs and errors as dirac_step. */
dirac_status dirac_run(dirac_op* op, void* psi_dev, void* hist_dev, int* n_hist, int n_steps,
                       double t_start, int* iters_out, double* resid_out);

/* Batched solve (the multi-instance form of the step, Sec. 2.4 applied to many pulse parameter
 * sets and radial sizes): advance n_inst independent instances by n_steps each.  ops[i] is an
 * instance's operator (its own basis, pulse, radial size and, for overlap, its own stream given at
 * setup; all on the current device, no op twice), psi_dev[i] / hist_dev[i] its state (complex128[n_i])
 * and history (complex128[2 n_i]) on the device, n_hist[i] (in/out, nullable = all 0) the valid
 * history entries, t_start[i] its start time.  Each instance runs its captured step driver
 * (dirac_run) on its own stream, so the instances' kernels overlap on the GPU; window > 0 keeps at
 * most `window` instances in flight (0: all).  iters_out / resid_out (host, nullable) are
 * [n_inst][n_steps].  Results equal per-instance dirac_run calls bit for bit.  Synchronises every
 * instance's stream.  Returns the first failing instance's status (every instance is completed and
 * its outputs written first); DIRAC_E_ARG on bad arguments before anything runs. */
dirac_status dirac_solve_batch(dirac_op* const* ops, int n_inst, void* const* psi_dev, void* const* hist_dev,
                               int* n_hist, int n_steps, const double* t_start, int window, int* iters_out,
                               double* resid_out);

/* Schedule autotuner of dirac_solve_batch: for each candidate window cand[0..ncand) and each
 * schedule of the complex64 preconditioner (v = 0: one lane per channel, v = 1: one warp per
 * channel, the fastest warp schedule available: rotated lanes, else staged, else plain) it times one step of all instances (host clock around launch and completion) from the
 * current states, restoring the states and histories afterwards (it allocates 3 n_i complex128
 * scratch per instance).  The fastest window goes to *best_window and every op keeps the fastest
 * preconditioner schedule (results are identical up to the solver tolerance across schedules; the
 * captured drivers are re-captured).  ms_out (host, nullable, 2 ncand) receives each time at
 * [v ncand + c].  Same argument rules as dirac_solve_batch. */
dirac_status dirac_batch_tune(dirac_op* const* ops, int n_inst, void* const* psi_dev, void* const* hist_dev,
                              const int* n_hist, const double* t_start, const int* cand, int ncand,
                              int* best_window, double* ms_out);

/* Observables of a state (Sec. 4.3): out[0] = psi^H S psi, out[1] = psi^H H0 psi,
 * out[2] = |v_1s^T S psi_{kappa=-1, mu=+1/2}|^2 (ground-state population),
 * out[3] = sum over channels (kappa, mu) and bound states b of |v_b^T S_kappa psi_{kappa mu}|^2, the
 * bound-state population, v_b the eigenvectors of H0_kappa v = E S_kappa v with -c^2 < E < 0,
 * v^T S v = 1.  n_out <= 4.  The first call with n_out = 4 computes those eigenvectors (one dense
 * generalised eigensolve per kappa on the GPU, cuSOLVER; seconds at N = 1000) and keeps them with
 * the op (2 n1 doubles per bound state); it allocates, so it must not run inside a stream capture.
 * Synchronises the op's stream.  Errors: DIRAC_E_ARG (bad argument), DIRAC_E_NUMERIC (the
 * eigensolver failed), DIRAC_E_CUDA. */
dirac_status dirac_observables(dirac_op* op, const void* psi_dev, double* out, int n_out);

/* y = A_sign x with the coupling values assembled by the most recent dirac_apply or dirac_step
 * (no reassembly).  Same buffers and errors as dirac_apply. */
dirac_status dirac_apply_assembled(dirac_op* op, int sign, const void* x_dev, void* y_dev);

/* The operator of the mixed-precision inner solve alone: y = A_sign(t) x (Eq. solPsi with the
 * coupling of Eq. fullH) in complex64 arithmetic, exactly as the inner BiCGSTAB applies it --
 * FP32 copies of S and H0 per kappa, FP32 coupling values (precision 1: the FP32 rounding of the
 * FP64 assembly; precision 2: the hi words of the double-float assembly), and the kernel the
 * solve uses: the owner/gather passes for order-7 splines, the factorised apply when
 * dirac_op_set_factorised is on, else the per-row kernel.  Assembles the coupling values for t
 * first.  x_dev, y_dev: device complex64[n] (interleaved re, im floats, library order), must not
 * alias.  Synchronises the op's stream (it reads the error word of the bounded bulk-copy waits).
 * Errors: DIRAC_E_ARG (NULL, aliasing, sign not +-1, precision 0), DIRAC_E_CUDA. */
dirac_status dirac_apply32(dirac_op* op, int sign, double t, const void* x_dev, void* y_dev);

/* z = M^-1 r in complex64 with the inner solve's current preconditioner schedule
 * (dirac_op_set_schedule(op, 1, ...)), M = S + i dt/2 H0 (Eq. matrixM) factored in FP64 and rounded
 * to FP32.  r_dev, z_dev: device complex64[n], must not alias.  DIRAC_E_ARG for precision 0. */
dirac_status dirac_precond_apply32(dirac_op* op, const void* r_dev, void* z_dev);

/* The refinement residual of a step, r = A_-(t) psi - A_+(t) x (Eq. solPsi), computed as the step
 * computes it: precision 2 in double-float by the owner/gather passes (order-7 splines) or the
 * per-row residual kernel, precision 0 and 1 in FP64 (b = A_- psi, then r = b - A_+ x).
 * Assembles the coupling values for t first.  psi_dev, x_dev, r_dev: device complex128[n]; r_dev
 * must alias neither.  bnorm (host, nullable) receives ||A_- psi||_2 as the step's tolerance test
 * uses it (precision 2: from FP32 products).  Synchronises the op's stream.  Errors: DIRAC_E_ARG,
 * DIRAC_E_CUDA. */
dirac_status dirac_residual(dirac_op* op, double t, const void* psi_dev, const void* x_dev, void* r_dev,
                            double* bnorm);

/* Kernel-phase timers.  dirac_profile(op, 1) resets and starts timing every launch group with a
 * pair of CUDA events on the op's stream (0 stops); dirac_profile_read synchronises the stream and
 * returns, per phase, the summed milliseconds and the number of timed launch groups, plus the
 * number of kernel launches since the reset (counted whether or not timing is on).
 * Phases: DIRAC_PHASE_ASSEMBLE (pulse factors + coupling values), DIRAC_PHASE_APPLY (double
 * precision operator products), DIRAC_PHASE_PRECOND, DIRAC_PHASE_VECTOR (updates, reductions,
 * copies), DIRAC_PHASE_APPLY32 (complex64 operator products of the mixed-precision inner solve),
 * DIRAC_PHASE_GUESS (the learned initial guess: features, network, correction), DIRAC_PHASE_OWNER
 * (the owner pass of the double-float refinement residual alone; also counted in
 * DIRAC_PHASE_APPLY, which covers the whole pass). */
#define DIRAC_PHASE_ASSEMBLE 0
#define DIRAC_PHASE_APPLY 1
#define DIRAC_PHASE_PRECOND 2
#define DIRAC_PHASE_VECTOR 3
#define DIRAC_PHASE_APPLY32 4
#define DIRAC_PHASE_GUESS 5
#define DIRAC_PHASE_OWNER 6
#define DIRAC_NPHASE 7
dirac_status dirac_profile(dirac_op* op, int enable);
dirac_status dirac_profile_read(dirac_op* op, double* ms, int64_t* count, int64_t* launches);

/* dirac_observables with no allocation in the call (the paper has no counterpart).  It serves
 * callers that cannot allocate GPU memory when they read the observables: real-time or monitoring
 * threads that must not hit the implicit device synchronisation of cudaMalloc/cudaFree, and
 * processes whose device footprint is fixed once setup is done.  Same arguments, outputs and errors
 * as dirac_observables, except n_out <= 3 (the bound-state population needs its eigenvectors set
 * up, which allocates).  Its scratch (block partials and the final sums) is a library-static device
 * array of 2 DIRAC_STATIC_MAX_PARTIALS + 2 complex128 values (about 2 MB): the driver allocates it
 * when it loads the library's module on a device (at the module's first use there, at the latest in
 * dirac_operator_setup), and that GPU holds it until the process exits.  dirac_operator_setup looks
 * up the array's device address (cudaGetSymbolAddress, with the op's device current), so this call
 * does no set-up; the address is kept for the life of the process, so the library must not be used
 * across a cudaDeviceReset.  It supports systems with channels x ceil((N+1)/128) <=
 * DIRAC_STATIC_MAX_PARTIALS and returns DIRAC_E_ARG beyond that, DIRAC_E_ARG for n_out outside 1..3,
 * DIRAC_E_STATE if the current device is not the op's, and DIRAC_E_STATE, with nothing enqueued, if
 * the op's stream is being captured into a CUDA graph (the call synchronises that stream).  All calls share the one array, which
 * keeps the last call's contents (every slot a call reads is written earlier in the same call):
 * calls whose work overlaps on the GPU (other streams, other host threads on the same device) race
 * on it and must be serialised by the caller.  It calls no cudaMalloc, cudaFree or other allocating
 * routine, and it synchronises the op's stream before returning the values. */
#define DIRAC_STATIC_MAX_PARTIALS 65536
dirac_status dirac_observables_static(dirac_op* op, const void* psi_dev, double* out, int n_out);

/* ---- Learned initial guess (no counterpart in the paper: it only changes where BiCGSTAB starts;
 * the solver's residual test still decides convergence, so the converged step is unchanged) ----
 * Per position p = (channel, radial slot): D_0..D_3 = backward differences of psi_n .. psi_{n-3}
 * at p (4 reals each: Re, Im of both DKB types), m_k their rms, s = m_3; features x[p] = [D_k / m_k
 * (16), clip(log10(m_j / m_3), -30, 30) / 10 for j = 0..2 (3), field factors at t_{n+1} (6: A0 wt_c
 * sin, cos of w_c (t - t0) for the three carriers of the sin^2 pulse, zero outside the pulse),
 * kappa / 10, 2 mu / 20, zeros] (32 floats; zero entries where an m is 0); the network a1 = tanh(x W1 + b1), a2 = tanh(a1 W2 + b2),
 * a3 = tanh(a2 W3 + b3), out = a3 W4 + b4 (W1 32 x 256, W2, W3 256 x 256, W4 256 x 4, weights
 * rounded to bfloat16 in every product, FP32 accumulation); guess = 3 psi_n - 3 psi_{n-1} + psi_{n-2}
 * + s out.  Parameters are one float array in the order W1, b1, W2, b2, W3, b3, W4, b4 (row-major
 * [in][out]); dirac_guess_param_count() gives its length.  Calls run on `stream` (NULL: the legacy
 * default stream) unless they take an op, whose stream they use. */
int64_t dirac_guess_param_count(void);
/* max_batch: largest training batch (sizes the training workspace, 6 max_batch x 256 floats). */
dirac_status dirac_guess_create(int max_batch, dirac_guess** out);
void dirac_guess_free(dirac_guess* net);
/* Copy parameters in (host, count = dirac_guess_param_count(); resets the optimiser) or out. */
dirac_status dirac_guess_set_params(dirac_guess* net, const float* host, int64_t count);
dirac_status dirac_guess_get_params(dirac_guess* net, float* host, int64_t count);
/* Features of every position of the op's system: states[0..3] = psi_n, psi_{n-1}, psi_{n-2},
 * psi_{n-3} (device complex128[n]); x_dev float[nch n1][32], s_dev float[nch n1] (device). */
dirac_status dirac_guess_features(dirac_op* op, const void* const* states, double t_next, float* x_dev,
                                  float* s_dev);
/* Training targets (psi_{n+1} - x_ext) / s: states[0..2] = psi_n, psi_{n-1}, psi_{n-2}, psi_next =
 * psi_{n+1}; t_dev float[nch n1][4]. */
dirac_status dirac_guess_targets(dirac_op* op, const void* const* states, const void* psi_next, const float* s_dev,
                                 float* t_dev);
/* out_dev float[M][4] = net(x_dev[M][32]).  tensor_cores 1: the bf16 kernel on the fifth-generation
 * tensor cores (tcgen05.mma, FP32 accumulators in tensor memory; the kernel the learned guess of a
 * step uses; this call then synchronises the stream to read the error word of its bounded waits and
 * returns DIRAC_E_CUDA if one ran out); 2: the bf16 warp-level mma.sync kernel (same arithmetic up
 * to FP32 summation order); 0: the FP32 kernels of training (batches of max_batch).  Input and
 * activations are rounded to bfloat16 on the tensor-core paths.  DIRAC_E_ARG for other values. */
dirac_status dirac_guess_forward(dirac_guess* net, const float* x_dev, int64_t M, float* out_dev, int tensor_cores,
                                 void* stream);
/* Mean squared error over B samples (0 < B <= max_batch) and, if grad_host != NULL, its gradient
 * (host float[param_count], gradient with respect to the rounded weights); synchronises. */
dirac_status dirac_guess_loss_grad(dirac_guess* net, const float* x_dev, const float* t_dev, int B, double* loss,
                                   float* grad_host, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the FP32 parameters from
 * the batch's gradient; loss (nullable) receives the batch loss before the step (synchronises). */
dirac_status dirac_guess_train_step(dirac_guess* net, const float* x_dev, const float* t_dev, int B, double lr,
                                    double* loss, void* stream);
/* Attach a network (not owned; NULL detaches) to an op: dirac_step with solver option guess = 2 then
 * starts each step from the network's guess once three past states are in the history, which must
 * then hold 3 n entries (psi_{n-1}, psi_{n-2}, psi_{n-3}; n_hist up to 3); before that the
 * extrapolated guess is used.  dirac_run and dirac_solve_batch do the same inside the captured
 * graph (their history buffers then hold 3 n entries too); results equal dirac_step's bit for bit. */
dirac_status dirac_op_set_guess(dirac_op* op, dirac_guess* net);

/* Overlapped assembly (precision 2 only; no counterpart in the paper, a scheduling choice): with
 * enable != 0, dirac_step assembles step s + 1's coupling values (they depend only on the time) on a
 * second stream into a second buffer set while step s solves, instead of at the start of step s + 1.
 * Results are identical (same kernels on the same data).  The first call allocates the second set
 * (the coupling values, K bands and pulse factors again: about the operator's coupling storage)
 * and a stream.  dirac_run and dirac_solve_batch do not overlap.  DIRAC_E_ARG if precision != 2. */
dirac_status dirac_op_set_overlap(dirac_op* op, int enable);

/* Accumulation of the double-float refinement residual's coupling sums (precision 2, order-7
 * splines; Eq. solPsi's r = A_- psi - A_+ x): mode 1 the Dot2 form (ten FP32 operations per
 * double-float multiply-add, error of order 2^-48 times each running sum); mode 2 the fixed-binade
 * form (six operations: every accumulator starts from an offset 1.5 * 2^k with 2^(k-2) at least a
 * bound of its sum of |products|, formed each pass from the coupling's static envelopes, the
 * pulse factors and the current vectors; error of order 2^-48 times the offset, so about
 * 1e-13 ||b|| on strong-field random states); mode 0 (the default) takes mode 2 when the solver
 * tolerance is at least 1e-11 and mode 1 below.  Both end on the same accurate residual test.
 * DIRAC_E_ARG for other modes. */
dirac_status dirac_op_set_residual_mode(dirac_op* op, int mode);

/* Preconditioner schedule of the complex128 (complex64 = 0) or complex64 (complex64 = 1) solve:
 * 0 one lane per channel (complex64 only; the channels of one kappa share the factor rows),
 * 1 one warp per channel, 2 one warp per channel with the vector and the factor rows staged
 * through shared memory, 3 one warp per channel with each row fixed to one lane (one shuffle
 * round per row; only factor chunks in shared memory, so every channel's warp is resident at
 * once).  dirac_operator_setup times the available ones and keeps the fastest; this call
 * overrides it (DIRAC_E_ARG if the schedule is not available for the op).  Schedules 1, 2 and 3
 * perform the same operations in the same order; 0 rounds differently (within the solver
 * tolerance). */
dirac_status dirac_op_set_schedule(dirac_op* op, int complex64, int sched);
int dirac_op_get_schedule(const dirac_op* op, int complex64);   /* -1 for a NULL op */

/* Factorised complex64 apply for the inner solve (precision 2, order-7 splines; Sec. 2.2 Eq. fullH):
 * the coupling is applied from the time-dependent radial bands and the angular coefficients (four
 * band products per channel and multipole, combined per pair) instead of the stored coupling
 * values.  Same operator; FP32 rounding differs, within the inner tolerance.  enable: 0 the stored
 * coupling (the default), 1 the subgroup form (products combined per 8 outputs of one mu, the
 * radial pass of the next tile beside the angular pass of the current one: the faster form at the
 * production size), 2 the per-channel form.  The first switch to a form builds its tables on the
 * host and allocates the products of two radial tiles (2 x channels x multipoles x 4 x 64 x 2
 * complex64) and, for form 1, the FP32 hi words of the radial bands (written by every later
 * assembly) and the subgroup item tables.  DIRAC_E_ARG for other precisions, spline orders or
 * modes; DIRAC_E_CUDA if the subgroup form's shared-memory need exceeds the device's limit.  The
 * input and output vectors of an apply must not alias. */
dirac_status dirac_op_set_factorised(dirac_op* op, int enable);

/* Self-test of the bounded waits of the owner passes (their bulk-copy rings): one block waits
 * limit_cycles SM clocks (at most 4e9, about two seconds) on an mbarrier phase that nothing
 * completes, records the time-out in the op's error word exactly as those passes do, and
 * *timed_out receives it (1 expected; the word is cleared again).  The context stays usable.
 * Synchronises the op's stream.  DIRAC_E_ARG on bad arguments. */
dirac_status dirac_selftest_wait(dirac_op* op, double limit_cycles, int* timed_out);

/* Differential photoelectron energy spectrum (Sec. 4.3, Eq. dPdE) of the device state psi_dev
 * (complex128, the library's layout, length n as in dirac_step):
 *   dP/dE = sum over the channels (kappa, mu) of |<psi_{kappa mu E} | psi>|^2.
 * The continuum states of a kappa are its eigenvectors v_j of H0_kappa v = E S_kappa v with
 * e_lo < E_j <= e_hi (v^T S v = 1); dividing by the square root of the local level spacing dE_j
 * (central difference of the neighbouring levels, one-sided at the window's ends) energy-normalises
 * them, so at a kappa's levels its density is sum over mu |v_j^T S psi_{kappa mu}|^2 / dE_j.
 * dpde[g] (host, n_grid doubles) = the sum over kappa of those densities linearly interpolated at
 * e_grid[g] (host; zero outside a kappa's first and last level in the window; a kappa with fewer
 * than two levels there adds nothing).  counts (may be NULL) receives two numbers: the levels in
 * the window over every kappa in use, and the projections formed (the sum over the channels of
 * their kappa's levels).  Energies in the shifted convention (bound states below 0).
 * The first call for a window computes the eigenpairs (cuSOLVER, per kappa; allocates, so not
 * inside a stream capture) and keeps them on the op; later calls with the same window reuse them.
 * Synchronises the op's stream.  DIRAC_E_ARG for a NULL op or state, non-finite or empty windows
 * (e_lo >= e_hi), n_grid < 0 or > 2^26, NULL grid arrays with n_grid > 0 or non-finite grid
 * energies; DIRAC_E_NUMERIC if the eigensolver fails. */
dirac_status dirac_spectrum(dirac_op* op, const void* psi_dev, double e_lo, double e_hi, int n_grid,
                            const double* e_grid, double* dpde, int64_t* counts);

/* Error of a spectrum against a reference (Sec. 4.3): *err = integral over [e1, e2] of
 * |p_n(E) - p_m(E)|^2 dE by the trapezoid rule over the grid points inside [e1, e2].  Host arrays of
 * n_grid doubles, e_grid strictly ascending.  DIRAC_E_ARG on NULL arrays, e1 > e2 or a grid that
 * does not ascend.  No GPU work. */
dirac_status dirac_spectrum_error(int n_grid, const double* e_grid, const double* p_n, const double* p_m,
                                  double e1, double e2, double* err);

/* Index-check word of a debug build (the library compiled with -DDG_BOUNDS): the owner and gather
 * passes and the grouped assembly test every computed global index of the coupling values, the
 * vectors and the partial products against the buffers' sizes before using it, skip the access
 * (or copy from the buffer's start) when it fails and set bit k of the word for check site k
 * (0 coupling rows of a copy, 1 vector window of a copy, 2 partial store, 3 partial read, 4
 * assembled coupling store).  *word receives the bits seen since the last call (then cleared);
 * *checked is 1 in a debug build, 0 in a release build (where the word stays 0).  Synchronises
 * the op's stream.  DIRAC_E_ARG on NULL arguments. */
dirac_status dirac_bounds_word(dirac_op* op, unsigned int* word, int* checked);

const char* dirac_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
