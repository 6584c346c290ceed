/*
 * dgls.h -- C ABI of libdgls.so: matrix-free DG0/DG1 residual, Jacobian-vector product,
 * Newton-GMRES implicit Euler step and adaptive discharge of the coarse-grained Li-S cathode
 * model of Okraschevski et al., "Structure Matters" (arXiv 2511.05233), on one NVIDIA GB300.
 *
 * Model: Tab. 4 (coarse-grained PDE system) with the Tradeoff Chemistry of Tab. 3, the
 * constitutive laws of Eqs. 2-6 and 18-24, Eq. 57 localisation, boundary conditions Eqs. 25-27;
 * discretisation Eqs. 43-48 (DG0 = two-point harmonic flux, DG1 = Q1 interior penalty);
 * time stepping Eq. 50; controllers Fig. 4 (naive) and Eqs. 51-54 (H211b); initial state
 * Tab. 6 and the parabolic relaxation of Sec. 2.8; cell voltage Eq. A1.
 *
 * Conventions for every call
 *  - All state vectors are FP64 arrays in device memory ("_dev") owned by the caller, laid out
 *    as dg_layout() reports: fields one after another; liquid fields and Phi^L have one value
 *    per voxel (index i + nx*(j + ny*k), x fastest), solid fields and Phi^S one value per
 *    structure voxel in increasing voxel index; DG1 stores 8 nodal values per voxel node-major
 *    (offset + node*len + voxel, node = a + 2b + 4c for the x, y, z Gauss-node indices).
 *  - Device calls are issued on the stream given to dg_setup and are asynchronous unless the
 *    comment says "synchronous".  No call aborts the process: errors are returned as a
 *    dg_status and described by dg_last_error().
 *  - The context owns its Krylov, preconditioner and scratch workspaces (allocated in
 *    dg_setup, freed in dg_destroy); it never takes ownership of caller buffers.
 */
#ifndef DGLS_H
#define DGLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DG_OK = 0,
    DG_ERR_ARG = -1,        /* invalid argument or structure */
    DG_ERR_OOM = -2,        /* workspace exceeds hbm_budget_bytes or cudaMalloc failed */
    DG_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    DG_ERR_NOCONV = -4,     /* Newton did not converge (iteration limit or line search) */
    DG_ERR_NONFINITE = -5,  /* NaN/Inf in a residual or update */
    DG_ERR_TIMEOUT = -6,    /* a bounded device-side wait gave up */
    DG_ERR_ABORTED = -7     /* time-step controller gave up (31st consecutive halving) */
} dg_status;

typedef struct dg_ctx dg_ctx;

/* Voxel structure (Sec. 2.1): phase per voxel, 0 macro-pore, 1 coarse-grained active
 * structure, 2 homogeneous separator.  x is the transport direction: the current collector is
 * the x = 0 face, the lithium anode the x = nx face.  dg_setup copies the array. */
typedef struct {
    int32_t nx, ny, nz;
    double h;                  /* voxel width in m */
    const uint8_t* phase;      /* host pointer, nx*ny*nz bytes, x fastest */
} dg_structure;

typedef enum { DG_CHEM_REDUCED3 = 0, DG_CHEM_TRADEOFF = 1 } dg_chemistry;
typedef enum { DG_PREC_FP64 = 0, DG_PREC_MIXED = 1 } dg_precision;

typedef struct {
    int32_t order;             /* 0: DG0 (Eq. 48), 1: DG1 tensor-product Q1 (Eqs. 43-47) */
    int32_t chemistry;         /* dg_chemistry: three-species (Li+, S8(L), S8^2-, E1 only, solids
                                  frozen) or the paper's Tradeoff Chemistry (Tab. 3) */
    double T;                  /* K; 298.15 reproduces Tab. 5.2 */
    double f_C;                /* discharge rate in 1/h (App. B, Eq. 18) */
    double j_el;               /* A/m^2; <= 0 derives j_el = f_C c_theo m_A,S8 (App. B) */
    double eps_struct;         /* structure fraction of the cathode, 1 - macro-porosity (Eq. 57) */
    double penalty;            /* DG1 interior-penalty factor (Eq. 46: 1) */
    int32_t smooth;            /* 1: rates of C2 and E4 multiplied by T_H(t) (Sec. 2.8, Eq. 56) */
    /* Newton-Krylov solver (the role of PETSc newtonls + gmres, Sec. 2.7) */
    int32_t precision;         /* dg_precision: FP64 Krylov, or FP32 JVP/basis/preconditioner
                                  inside the FP64 Newton iteration */
    int32_t gmres_restart;     /* Krylov subspace size m (30) */
    int32_t gmres_max_it;      /* total GMRES iterations per linear solve */
    double newton_rtol;        /* converged when ||S R|| <= max(rtol ||S R(z^n)||, atol sqrt(n_dof)) */
    double newton_atol;        /* RMS floor of the scaled residual (1e-12): just above its rounding
                                  level, which a nearly converged step (a late relaxation step) reaches */
    int32_t newton_max_it;     /* 25 */
    double eta_max;            /* Eisenstat-Walker forcing-term cap (1e-2) */
    double eta_min;            /* forcing-term floor (1e-3): keeps the middle Newton iterations from
                                  over-solving; the last iteration's tolerance still follows from
                                  newton_rtol, and convergence is tested on the true residual */
    int64_t hbm_budget_bytes;  /* workspace cap checked in dg_setup (0: no cap) */
    int32_t preconditioner;    /* 0: cell-block Jacobi; 1: two-stage (CPR): multigrid on the potential
                                  block, then block Jacobi on the remainder; 2: the additive form of the
                                  same two levels, no Jacobian-vector product inside (default) */
    int32_t mg_cycles;         /* V-cycles of the potential multigrid per application (1; 1 to 16): a later cycle
                                  starts from the current iterate of the finest level */
    int32_t precond_every;     /* rebuild the preconditioner every k-th Newton iteration of a step
                                  (0: once per step, at its first iteration) */
    double newton_stall_rtol;  /* a Newton solve whose line search can no longer reduce ||S R||, or whose
                                  last iteration reduced it by less than half, counts as converged if
                                  ||S R|| <= newton_stall_rtol ||S R(z^n)|| (1e-8, PETSc's default
                                  relative tolerance): at large dt the FP64 rounding level of the
                                  scaled residual lies above newton_rtol ||S R(z^n)|| */
    int32_t reorth;            /* classical Gram-Schmidt in GMRES: 2 = one pass (PETSc's default GMRES
                                  orthogonalisation, the solver of Sec. 2.7; default); 0 = a second
                                  pass when the first cancelled, ||w'|| < ||w|| / sqrt(2)
                                  (Daniel-Gragg-Kaufman-Stewart); 1 = always two passes (CGS2) */
    int32_t species_mg;        /* with preconditioner 1 or 2: coarse correction of the liquid species rows
                                  (an aggregation multigrid per pair of species on P^T S J P, P the
                                  voxel-constant prolongation: the storage and own-species reaction
                                  diagonal plus the diffusion conductances of Eq. 48, or of the interior
                                  penalty of Eq. 46 for DG1), applied together with the potential
                                  correction in the multiplicative form (one more Jacobian-vector product
                                  per application).  0 = off; 1 = on; 2 = on when
                                  max_m D_m^0 dt / h^2 >= 10, the steps where diffusion reaches past
                                  the neighbouring voxels (default) */
    int32_t jvp_form;          /* DG1 Jacobian-vector products inside the Krylov loop: 0 = automatic
                                  (fused for an FP32 Krylov loop, cached linearisation for FP64;
                                  default); 1 = cached linearisation (node Jacobians and face data,
                                  built once per Newton iteration); 2 = fused matrix-free kernel
                                  (dual numbers, one launch, nothing cached) */
} dg_params;

typedef struct {
    int32_t converged;         /* 1 if Newton converged */
    int32_t newton_iterations;
    int32_t gmres_iterations;  /* summed over Newton iterations */
    int32_t residual_evals;
    int32_t jvp_evals;
    double norm0, norm;        /* scaled residual norms ||S R|| at start and end */
} dg_step_info;

typedef enum { DG_CTRL_NAIVE = 0, DG_CTRL_H211B = 1, DG_CTRL_FIXED = 2 } dg_controller;

/* Controller state between two calls of dg_discharge (checkpoint / resume).  Together with the
 * state vector it is everything the discharge loop carries from one accepted step to the next,
 * so a run split at any accepted step and resumed from this record and the state continues
 * bitwise as the uninterrupted run (all reductions have a fixed order). */
typedef struct {
    double t;                  /* time of the state, s */
    double dt;                 /* step size of the next attempt, s */
    double err_prev, dt_prev;  /* H211b filter history (Eq. 51): last accepted error and step */
    int32_t sct;               /* naive controller (Fig. 4): successes since the last growth */
    int32_t halvings;          /* consecutive halvings so far */
} dg_controller_state;

typedef struct {
    int32_t controller;        /* dg_controller */
    double t0, dt0, dt_min, dt_max;
    double tol;                /* H211b tolerance (Eq. 51) */
    double cutoff_V;           /* stop at the first accepted step with U_cell <= cutoff (1.9 V) */
    double t_end;              /* stop when t >= t_end (<= 0: no limit) */
    int32_t max_steps;         /* accepted-step limit */
    int32_t max_halvings;      /* consecutive halvings before DG_ERR_ABORTED (30) */
    const double* replay_dt;   /* host array: if non-NULL take these step sizes (n_replay) */
    int32_t n_replay;
    int32_t limiter;           /* DG1: 1 applies dg_limit to the state after every accepted step */
    const dg_controller_state* resume;  /* non-NULL: continue a checkpointed run; its t and dt
                                           replace t0 and dt0 */
} dg_discharge_opts;

typedef struct {               /* caller-allocated host arrays of length n_max */
    int32_t n_max;
    int32_t n;                 /* accepted steps written */
    double* t;                 /* time after the step, s */
    double* dt;                /* accepted step size, s */
    double* U_cell;            /* Eq. A1, V */
    double* c_m;               /* c_m = t f_C c_theo, Ah/kg (App. B) */
    int32_t* newton_its;       /* per accepted step */
    int32_t* gmres_its;
    int32_t status;            /* dg_status of the run: DG_OK (cut-off, t_end or max_steps) */
    int32_t attempts, failures;
    dg_controller_state* checkpoint;  /* non-NULL: receives the controller state when the call
                                         returns (pass it as opts.resume with the returned state) */
} dg_curve;

/* Default parameters of the paper (Tabs. 1, 2, 5) for a chemistry and DG order. */
dg_status dg_params_default(dg_params* p, int32_t chemistry, int32_t order);

/* Copy the structure, build the compacted structure list and neighbour data, upload the
 * parameters and allocate the workspaces on `cuda_stream` (NULL: legacy default stream).
 * DG_ERR_ARG if no structure voxel touches the current collector or the anode layer is not
 * liquid; DG_ERR_OOM if the workspace exceeds hbm_budget_bytes.  Synchronous. */
dg_status dg_setup(const dg_structure* s, const dg_params* p, void* cuda_stream, dg_ctx** out);

/* Device bytes that dg_setup_in needs for this structure and these parameters (every workspace the
 * context holds, each on a 256-byte boundary), computed without allocating or touching the device
 * (no counterpart in the paper: it sizes admission and buffer reuse in a server).  DG_ERR_ARG as
 * dg_setup.  Host only. */
dg_status dg_workspace_estimate(const dg_structure* s, const dg_params* p, int64_t* bytes);

/* dg_setup with every workspace carved from the caller's device buffer workspace_dev (256-byte
 * aligned, workspace_bytes long, at least dg_workspace_estimate's bytes; DG_ERR_OOM if smaller) instead
 * of cudaMalloc, so that a caller can keep a buffer and reuse it for the next context once this one is
 * destroyed.  The caller owns the buffer and must keep it allocated until dg_destroy.  Synchronous. */
dg_status dg_setup_in(const dg_structure* s, const dg_params* p, void* cuda_stream, void* workspace_dev,
                      int64_t workspace_bytes, dg_ctx** out);
dg_status dg_destroy(dg_ctx* ctx);
const char* dg_last_error(const dg_ctx* ctx);

/* Number of unknowns and per-field offset/length (lengths include the 8 DG1 nodes).
 * Arrays hold up to 10 entries; *n_fields receives 10 (Tradeoff) or 5 (three-species). */
dg_status dg_layout(const dg_ctx* ctx, int64_t* n_dof, int32_t* n_fields,
                    int64_t field_offset[10], int64_t field_len[10]);

/* Tab. 6 equilibrium written into z_dev (Phi^L = 0, Phi^S = Delta Phi_0; three-species:
 * 1000/10/100 mol/m^3 and the Nernst potential of E1).  Asynchronous. */
dg_status dg_equilibrium_state(dg_ctx* ctx, double* z_dev);

/* Parabolic relaxation of Sec. 2.8 applied to z_dev in place: n_steps implicit Euler steps of
 * size dt with concentrations frozen, d_t Phi terms and the current ramped by T_H.  Synchronous. */
dg_status dg_relax(dg_ctx* ctx, double* z_dev, double dt, int32_t n_steps);

/* Residual R(z; z^n, t, dt) of the implicit Euler step (Eq. 50) in the DG weak form,
 * volume-integrated, unscaled.  t is the time at which T_H is evaluated (t^{n+1}).
 * z_dev, zold_dev, r_dev: n_dof doubles; r_dev must not alias the inputs.  Asynchronous. */
dg_status dg_residual(dg_ctx* ctx, const double* z_dev, const double* zold_dev,
                      double t, double dt, double* r_dev);

/* Allocation-free variant of dg_residual for DG0 contexts (the paper has no counterpart: this
 * serves callers of this library).  It is for code that may not allocate device memory when it
 * runs -- inside CUDA stream capture, where cudaMalloc is illegal, or in a process whose device
 * memory belongs to an external allocator -- and that must leave the context's own workspaces
 * untouched: it reads the context's geometry and parameters only and keeps its scratch (one
 * transport factor per voxel) in a static device array of 2,097,152 doubles (16 MiB, 128^3
 * voxels) that every GPU loading the library holds until the process exits.  Larger grids and
 * DG1 contexts return DG_ERR_ARG with a message in dg_last_error().  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Every call shares the array and overwrites
 * all of it that it reads, so nothing needs clearing, but two calls that overlap on the GPU
 * (different streams or threads) race on it.  Inputs, output and asynchrony as dg_residual. */
dg_status dg_residual_noalloc(dg_ctx* ctx, const double* z_dev, const double* zold_dev,
                              double t, double dt, double* r_dev);

/* Jacobian-vector product J(z) v with J = dR/dz at fixed z^n, t, dt (exact forward-mode
 * linearisation of dg_residual).  Asynchronous. */
dg_status dg_jvp(dg_ctx* ctx, const double* z_dev, double t, double dt,
                 const double* v_dev, double* jv_dev);

/* Jacobian-vector product J(z) v of dg_jvp by the matrix-free kernels the Krylov loop of a
 * mixed-precision context runs (forward-mode dual numbers, nothing cached; Eqs. 43-48 with the
 * Tab. 4 system): for DG1 the fused kernel, one launch that reads z and v once and writes J v once;
 * for DG0 the two-launch product (transport factors, then voxels).  precision DG_PREC_FP64: v_dev
 * and jv_dev are n_dof doubles and the arithmetic is FP64; DG_PREC_MIXED: they are n_dof floats, z
 * is rounded to FP32 on the device and the arithmetic is FP32 (the context must have been set up
 * with precision DG_PREC_MIXED, which holds the FP32 copy of z).  The FP32 arithmetic uses the
 * hardware exponential, logarithm, reciprocal and square root; its element-wise error against the
 * exact product stays below 2e-5 |J||v| (the tested bound).  Rows unscaled, as dg_jvp.
 * Asynchronous. */
dg_status dg_jvp_fused(dg_ctx* ctx, const double* z_dev, double t, double dt, int32_t precision,
                       const void* v_dev, void* jv_dev);

/* Apply the cell-block-Jacobi preconditioner built at z: out = B(z)^{-1} v, where B holds the
 * diagonal blocks of S J (S the Newton row scales; DG0 full voxel blocks, DG1 per-node field
 * blocks).  Asynchronous. */
dg_status dg_block_jacobi(dg_ctx* ctx, const double* z_dev, double t, double dt,
                          const double* v_dev, double* out_dev);

/* Newton row scale of every unknown (dt/(M c_ref) for species and solids, dt/(M F c_ref) for
 * the potentials, M the voxel or node volume) written to s_dev.  Asynchronous. */
dg_status dg_row_scales(dg_ctx* ctx, double dt, double* s_dev);

/* One implicit Euler step (Eq. 50) from z^n at time t to t + dt by Newton-GMRES with
 * block-Jacobi right preconditioning.  zn_dev is read, z_dev receives z^{n+1} (they may be
 * the same buffer).  On DG_ERR_NOCONV z_dev holds the last Newton iterate.  Synchronous. */
dg_status dg_step(dg_ctx* ctx, const double* zn_dev, double* z_dev, double t, double dt,
                  dg_step_info* info);

/* Same step with host buffers: copies zn_host to the device, steps, copies z^{n+1} back to
 * z_host.  Synchronous. */
dg_status dg_step_host(dg_ctx* ctx, const double* zn_host, double* z_host, double t, double dt,
                       dg_step_info* info);

/* Cell voltage U_cell (Eq. A1): mean of Phi^S over the structure faces at x = 0. Synchronous. */
dg_status dg_cell_voltage(dg_ctx* ctx, const double* z_dev, double* U_cell);

/* Ledger (Eq. A3 numerators and Sec. 3.2 conservation): out[0] total dissolved + solid sulfur
 * (mol), out[1] total lithium (mol), out[2] liquid charge (C), out[3] Phi^L mean over the anode
 * face, out[4] Phi^L mean over the x = 0 face.  Synchronous. */
dg_status dg_ledger(dg_ctx* ctx, const double* z_dev, double out[5]);

/* Galvanostatic discharge from z_dev (in place) under the chosen controller until the
 * cut-off voltage, t_end or max_steps; one curve point per accepted step.  With
 * out->checkpoint the controller state at return is written there; with opts->resume the run
 * continues from such a record (checkpoint / resume of a long discharge).  Synchronous. */
dg_status dg_discharge(dg_ctx* ctx, double* z_dev, const dg_discharge_opts* opts, dg_curve* out);

/* Kernel timing by category, recorded with CUDA events on the context stream while enabled:
 * 0 residual, 1 Jacobian-vector product, 2 preconditioner build, 3 preconditioner apply,
 * 4 Krylov orthogonalisation and updates.  dg_profile(ctx, 1) clears and enables, 0 disables;
 * dg_profile_read fills ms[5] (summed device milliseconds) and launches[5] (calls). */
dg_status dg_profile(dg_ctx* ctx, int32_t enable);
dg_status dg_profile_read(const dg_ctx* ctx, double ms[5], int64_t calls[5]);

/* Vertex-based slope limiter of App. B (Kuzmin's rule, which the paper applies to its DG1 scheme
 * because that scheme is not positivity-preserving, Sec. 2.6), in place on the liquid species of a
 * DG1 state z_dev.  Per voxel and species, the deviation of the conserved density q = eps_L c from
 * its voxel mean is scaled by the largest factor in [0, 1] that keeps the Q1 field's value at every
 * voxel corner within the range of the means of the voxels sharing that corner (only voxels inside
 * the domain).  Voxel means of q, hence all species amounts, are unchanged; non-negative means give
 * non-negative nodal concentrations.  Solid fractions and potentials are left alone.  DG_ERR_ARG for
 * DG0 contexts.  Asynchronous on the context's stream; uses the context's scratch. */
dg_status dg_limit(dg_ctx* ctx, double* z_dev);

/* ---- Batches: several independent cells (uneven grids, DG0 and DG1, one chemistry) evaluated
 * together (no counterpart in the paper, which runs one cell per job).  The products and the DG0
 * residual of all instances run as one launch per kind over the instances' concatenated blocks, with
 * each instance's parameters, geometry and buffers in device job records; the blocks go through the
 * same device functions as a single instance, so every instance gets the result it gets alone.  The
 * batch keeps its own launch stream; its calls use the contexts' scratch buffers, so a context must
 * not run work of its own while a batch call that contains it is in flight. */
typedef struct dg_batch dg_batch;

/* Batch of n contexts (all of one chemistry; DG_ERR_ARG otherwise) launching on cuda_stream (NULL:
 * legacy default stream).  Allocates the schedules and job records once.  The contexts stay owned
 * by the caller and must outlive the batch.  Synchronous. */
dg_status dg_batch_create(dg_ctx* const* ctxs, int32_t n, void* cuda_stream, dg_batch** out);
dg_status dg_batch_destroy(dg_batch* b);
const char* dg_batch_last_error(const dg_batch* b);
/* Kernels this batch has launched (monotone counter). */
int64_t dg_batch_launch_count(const dg_batch* b);

/* Per instance k: jv[k] = J_k(z[k]) v[k], the product dg_jvp_fused computes for that context (host
 * arrays of n device pointers and n times; precision as dg_jvp_fused, MIXED needs mixed contexts).
 * One launch for all DG1 instances, two for all DG0 instances (plus one FP32 rounding launch for
 * MIXED).  Asynchronous on the batch stream. */
dg_status dg_batch_jvp(dg_batch* b, const double* const* z_dev, const double* t, const double* dt,
                       int32_t precision, const void* const* v_dev, void* const* jv_dev);

/* Per instance k: r[k] = R_k(z[k]; zold[k], t[k], dt[k]) as dg_residual.  DG0 instances: two launches
 * for all; DG1 instances: each instance's own face-once kernels, issued on the batch stream.
 * Asynchronous on the batch stream. */
dg_status dg_batch_residual(dg_batch* b, const double* const* z_dev, const double* const* zold_dev,
                            const double* t, const double* dt, double* const* r_dev);

/* Schedule autotuner: times the batch's products on these inputs (one warm-up and three timed
 * launches per candidate, CUDA events on the batch stream) for each block order of the DG1 launch
 * (0: instance after instance, 1: one block of every instance in turn) and each block size of the
 * DG0 launches (64, 128, 256, 512 voxels), keeps the fastest for later calls and reports them in
 * choice[0] (DG1 order) and choice[1] (DG0 block size).  Overwrites jv.  Synchronous. */
dg_status dg_batch_autotune(dg_batch* b, const double* const* z_dev, const double* t, const double* dt,
                            int32_t precision, const void* const* v_dev, void* const* jv_dev, int32_t choice[2]);

/* One implicit Euler step of every instance (dg_step of each context, concurrently from host threads,
 * each on its own context's stream): status[k] receives dg_step's status, info[k] (if info) its
 * statistics.  Returns DG_OK unless the arguments are bad.  Synchronous. */
dg_status dg_batch_step(dg_batch* b, const double* const* zn_dev, double* const* z_dev, const double* t,
                        const double* dt, dg_step_info* info, int32_t* status);

/* Number of CUDA kernels this context has launched (monotone counter). */
int64_t dg_launch_count(const dg_ctx* ctx);

/* Second Gram-Schmidt passes GMRES has taken (monotone counter; with reorth = 1, one per
 * Arnoldi step). */
int64_t dg_reorth_count(const dg_ctx* ctx);

/* Workspace bytes held by the context on the device. */
int64_t dg_workspace_bytes(const dg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DGLS_H */
