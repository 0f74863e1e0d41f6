/*
 * mot.h — C ABI of the GB300 marching-on-in-time (MOT) library for the
 * Calderon-preconditioned, quasi-Helmholtz-regularised ("qHP") time-domain
 * PMCHWT equation of Le, Muenger, Andriulli, Cools, "A Stable, Accurate, and
 * Well-Conditioned Time-Domain PMCHWT Formulation" (arXiv 2510.07989).
 *
 * One MOT step solves Eq. (MOT):  Q_0 w_i = r_i - sum_{k>=1} Q_k w_{i-k},
 * with Q_k = Q_k^ll + Q_k^ls + Q_k^sl + Q_k^ss built from the lagged
 * interaction matrices of Section V-B, the static preconditioner
 * T = P^{Sigma H} T_0^s P^{Sigma H} + P^Lambda T_0^h P^Lambda (Eq. (CP)),
 * the Gram matrix G (Section III) and the quasi-Helmholtz projectors
 * (Section IV-B). Everything runs on one CUDA device (sm_103a).
 *
 * Conventions
 *   - All arrays are plain C arrays; "host" pointers are read during the call
 *     and never retained (the library copies what it needs).
 *   - Unknown layout for B right-hand sides: w[b][0][m] = u_m, w[b][1][m] = v_m,
 *     m in canonical edge order (see mot_create).
 *   - Floating point is IEEE binary64 unless stated.
 *   - Every function returns MOT_OK (0) or a negative status; no C++ exception
 *     crosses this boundary. mot_last_error() returns a message for the last
 *     failing call on a handle.
 *   - A handle is not thread safe; calls on one handle must be serialised.
 *     Distinct handles may be used from different host threads at once (the
 *     library's only shared mutable state is per-device kernel attributes,
 *     set once, and the staging array of mot_fields_noalloc, whose calls the
 *     caller serialises; mot_run_many relies on this).
 */
#ifndef MOT_H
#define MOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MOT_OK = 0,
    MOT_EINVAL = -1,   /* bad argument: sizes, NaN/Inf, K too small, open mesh ... */
    MOT_EOOM = -2,     /* device or host allocation failed */
    MOT_ENOCONV = -3,  /* GMRES or CG reached its iteration limit (result kept, flagged) */
    MOT_ECUDA = -4,    /* CUDA runtime error (message in mot_last_error) */
    MOT_ESTATE = -5    /* call out of order (e.g. step before load_operators) */
};

enum { MOT_PREC_FP64 = 0, MOT_PREC_MIXED = 1 };

typedef struct mot_handle mot_handle;

/* Closed, outward-oriented triangle mesh (paper Section II). */
typedef struct {
    int32_t nv;            /* number of vertices */
    const double* verts;   /* [nv][3] host */
    int32_t nf;            /* number of triangles */
    const int32_t* tris;   /* [nf][3] host, counter-clockwise seen from outside */
} mot_mesh;

/* Solver options; pass NULL for defaults. */
typedef struct {
    int32_t precision;     /* MOT_PREC_FP64 (default) */
    int32_t device;        /* CUDA device ordinal, default 0 */
    double gmres_tol;      /* relative residual of the Q_0 solve, default 1e-13 (FP64), 1e-11 (mixed) */
    int32_t gmres_maxit;   /* default 200 */
    double cg_tol;         /* relative residual of Laplacian / Gram solves, default 1e-14 */
    int32_t cg_maxit;      /* default 5000 */
    int32_t timing;        /* 1: time every history-contraction launch with CUDA events
                              on its stream (reported by mot_get_info); default 0 */
    int32_t mixed_flags;   /* MOT_PREC_MIXED only; 0 = default (MOT_MIX_DEFAULT). Bits:
                              MOT_MIX_HIST32: FP32 history tiles and panels
                              MOT_MIX_LF32:   FP32 dense left factor [M1 | M2]
                              MOT_MIX_Q032:   FP32 dense Q_0 in the GMRES iterations
                              MOT_MIX_REFINE: FP64 iterative refinement of the Q_0 solve
                              MOT_MIX_PRECOND: right-preconditioned GMRES with an FP32
                                 copy of Q_0^{-1} (LU with partial pivoting at load)
                              MOT_MIX_TC:     with MOT_MIX_HIST32, B a multiple of 8 and an
                                 sm_100-family GPU, the history contraction runs on the tensor cores
                                 (tcgen05): FP32 tiles and coefficients split into three
                                 bf16 slices each, FP32 accumulation, compensated sums
                              MOT_MIX_TCBULK: with MOT_MIX_TC, the bulk form of the tensor-core
                                 history: columns in one global order (instead of sorted per
                                 row block), coefficient panels kept pre-swizzled in 32-row
                                 blocks and moved by bulk copies (no per-row gather)
                              MOT_MIX_EMU64:  on an sm_100-family GPU, the FP64 dense products
                                 of the step (left factor, refinement residual) run on the
                                 tensor cores as exact products of 7-bit integer slices
                                 (relative error about 2^-40 of sum |A||x|) */
    int32_t refine_sweeps; /* MOT_MIX_REFINE: FP64 residual + correction sweeps per step
                              (stops early once |r| <= gmres_tol |b|); default 1 */
    int32_t fp64_precond;  /* MOT_PREC_FP64 only. 0 (default): GMRES on Q_0 in product form,
                              unpreconditioned. 1: right-preconditioned GMRES, Q_0 M z = b,
                              x = M z, with M = Q_0^{-1} formed at load in FP64 (Q_0 from the
                              product form on unit columns, LU with partial pivoting); every
                              product stays FP64, so the result matches the unpreconditioned
                              solve to the GMRES tolerance while the iteration count drops to
                              a few. Costs (2 npad)^2 doubles of device memory. */
    int32_t hist_stall_test; /* testing of the failure path only; 0 (default) = off. k > 0:
                              every tensor-core history launch withholds the copies of the
                              k-th pipeline stage of its first CTA (the k-th task with one
                              task per stage), whose pipeline waits then give up
                              after 1 ms; that CTA stops, drains its copies, releases TMEM
                              and raises the error word, and mot_step returns MOT_ECUDA
                              with the GPU context intact. */
    int32_t fp64_direct;   /* MOT_PREC_FP64 only. 0 (default): the Gram solves (G^{-1} in the
                              left factor) by CG on the normal equations and the projector
                              solves by CG on the graph Laplacians, to cg_tol. 1: by dense
                              FP64 inverses formed at load (LU with partial pivoting; the
                              Laplacians as (L + 11^T/N)^{-1}, their pseudo-inverse on the
                              mean-free right-hand sides), exact to rounding; costs
                              npad^2 + nf^2 + nv^2 doubles of device memory. */
} mot_options;

enum { MOT_MIX_HIST32 = 1, MOT_MIX_LF32 = 2, MOT_MIX_Q032 = 4, MOT_MIX_REFINE = 8, MOT_MIX_PRECOND = 16,
       MOT_MIX_TC = 32, MOT_MIX_EMU64 = 64, MOT_MIX_TCBULK = 128,
       MOT_MIX_DEFAULT = MOT_MIX_HIST32 | MOT_MIX_Q032 | MOT_MIX_REFINE | MOT_MIX_PRECOND | MOT_MIX_TC |
                         MOT_MIX_EMU64 };

/*
 * Lag-window sparse matrix (one family / medium of Section V-B):
 * for row m, entries e in [rowptr[m], rowptr[m+1]) hold column col[e] and
 * values val[voff[e] .. voff[e] + cnt[e] - 1] for lags k0[e] .. k0[e]+cnt[e]-1.
 * For K~ (Section V-B-3) tail_lag/tail_val (nullable otherwise) give a
 * constant tail_val[e] for lags tail_lag[e] .. k_max - 1.
 */
typedef struct {
    int64_t nent;
    const int64_t* rowptr;   /* [ne+1] */
    const int32_t* col;      /* [nent] */
    const int32_t* k0;       /* [nent] */
    const int32_t* cnt;      /* [nent] */
    const int64_t* voff;     /* [nent] */
    const double* val;       /* values */
    const int32_t* tail_lag; /* [nent] or NULL */
    const double* tail_val;  /* [nent] or NULL */
} mot_lagmat;

/*
 * Every input of the MOT step (host pointers, copied by mot_load_operators).
 *   mat[0..5]  exterior medium: A.T, A.K, Ah.T, Ah.K, At.T, At.K
 *   mat[6..11] interior medium: same order.
 *     A  : T_k, K_k        (h_0 basis, collocation at k dt; Section V-B-1)
 *     Ah : T^_k, K^_k      (T_max d/dt of q_0; Section V-B-2)
 *     At : T~_k, K~_k      ((1/T_max) d/dt^-1 of p_0; Section V-B-3)
 *   T0s, T0h : static BC-space operators T_0^s, T_0^h (Section III), dense
 *              row-major ne x ne.
 *   G  : Gram matrix <n x f_m, g_n> (Section III), CSR ne x ne.
 *   rhs_x, rhs_wf : RWG quadrature table [ne][nq][3] of points and
 *              weight * area * f_m(x) (both triangles of each edge), used to
 *              test the incident field (Section V-C) and for far fields.
 */
typedef struct {
    mot_lagmat mat[12];
    const double* T0s;
    const double* T0h;
    const int64_t* g_rowptr;
    const int32_t* g_col;
    const double* g_val;
    int32_t nq;
    const double* rhs_x;
    const double* rhs_wf;
} mot_operators;

/* Gaussian plane wave of Eq. (hin): amplitude A, polarisation p, direction k,
 * width w, arrival t0; the star right-hand side is forced to 0 for
 * i dt > t_trunc (Section V-C). */
typedef struct {
    double A;
    double p[3];
    double k[3];
    double w;
    double t0;
    double t_trunc;
} mot_wave;

typedef struct {
    int32_t ne, nv, nf;
    int32_t kmax;          /* ceil(T_max/dt) */
    int32_t K;             /* history lags used (k_max + 1) */
    int32_t B;             /* current batch size (0 before the first step) */
    int64_t step;          /* steps completed */
    double D, tmax, dt;
    int32_t last_gmres_iters;   /* max over the batch, last step */
    double last_gmres_resid;    /* max relative residual, last step */
    int32_t last_cg_iters;      /* max CG iterations of any projector/Gram solve, last step */
    int64_t device_bytes;       /* device memory held by the handle */
    int64_t gpu_launches;       /* kernels launched by this handle so far */
    double tile_fill;           /* nonzero fraction of the stored history tiles */
    int64_t tile_count;         /* stored history tiles (all lags and families) */
    /* algorithmic work of one full-depth history contraction (all lags live):
       2 flops per stored nonzero per right-hand-side column it multiplies,
       and per stored nonzero plus per coefficient of the lags it reads one
       value at the stored precision (8 bytes FP64, 4 bytes on the mixed path) */
    double hist_flops_per_step;
    double hist_bytes_per_step;
    /* with mot_options.timing: history-contraction launches (full depth, lags
       1..K) timed so far and their summed CUDA-event duration */
    int64_t hist_timed_launches;
    double hist_timed_ms;
    /* with mot_options.timing: summed CUDA-event time (ms) of the step phases:
       [0] right-hand side, [1] history contraction, [2] left factor,
       [3] Q_0 GMRES solve, [4] FP64 refinement, [5] projector + ring update,
       [6] current recovery and Fourier sums */
    double phase_ms[8];
    /* history kernel of the current batch: 0 FP64, 1 FP32 CUDA cores,
       2 tensor cores (tcgen05, bf16 x 3 slices) */
    int32_t hist_kernel;
    /* tensor-core history: tasks of one full-depth launch (each multiplies one
       gathered 32 x 2B coefficient panel by two 32 x 32 tiles) */
    int64_t hist_tc_tasks;
    /* GMRES iterations of the Q_0 solves summed over every step since the
       march (re)started (the refinement's correction solves excluded) */
    int64_t gmres_iters_total;
    /* tensor-core history: the configuration in use -- tasks per chunk, the
       fraction of the L2 one lag range of the task list may fill, pipeline
       stages (0: the deepest that fits) -- whether mot_tune (or mot_run_many)
       chose it, and its launch time in that tuning (ms) */
    int32_t tc_chunk_cap;
    double tc_lag_frac;
    int32_t tc_stages;
    int32_t tc_tuned;
    double tc_tune_ms;
    /* launches of the tensor-core history kernel that served this handle so far
       (steps, tuning trials, launches shared with other scatterers) */
    int64_t tc_launches;
    /* epilogue warps of the tensor-core history (4, or 8: two per TMEM lane
       quarter, one output each); a tuning choice like the three above */
    int32_t tc_epilogue_warps;
    /* tasks per pipeline stage of the tensor-core history (1, or 2: the stage
       holds two tasks' operands behind one full / empty barrier pair); a
       tuning choice like the others */
    int32_t tc_tasks_per_stage;
} mot_info;

/*
 * Create a solver for one scatterer (paper Section II).
 *   mesh   : closed 2-manifold, outward orientation. The library builds the
 *            canonical edge table: edges are vertex pairs (a<b) sorted
 *            lexicographically, oriented v^- = a -> v^+ = b; c^+ is the
 *            triangle left of that direction seen from outside.
 *   eps_r, mu_r : interior material relative to the exterior (c = 1, eta = 1).
 *   dt     : time step (> 0).
 *   K      : number of history lags to keep; must be >= k_max + 1 with
 *            k_max = ceil(T_max/dt), T_max = D / min(c, c') (Eq. (alpha)),
 *            D = largest vertex distance.
 * Errors: MOT_EINVAL (open/non-manifold mesh, eps_r/mu_r/dt <= 0, K too
 * small), MOT_ECUDA, MOT_EOOM. On success *out owns device memory until
 * mot_destroy.
 */
int mot_create(const mot_mesh* mesh, double eps_r, double mu_r, double dt, int K, const mot_options* opt,
               mot_handle** out);

/* Copy all operators to the device and build the internal block-sparse
 * layout. Errors: MOT_EINVAL (NaN/Inf, lag beyond its family's range,
 * index out of range), MOT_EOOM, MOT_ECUDA, MOT_ESTATE (called twice). */
int mot_load_operators(mot_handle* h, const mot_operators* ops);

/*
 * Optional: frequencies (angular, rad per unit time) of the running Fourier
 * transforms of the recovered loop and star currents (Eq. (dis_jm); the two
 * parts are accumulated separately). Must be called before the first step.
 */
int mot_set_frequencies(mot_handle* h, int n_freq, const double* omega);

/*
 * Advance one MOT step (Eq. (MOT): right-hand side of Section V-C, history
 * sum over the lags, Q_0 solve, loop/star ring update, current recovery of
 * Eq. (dis_jm)) for B plane waves (B <= 64, fixed after the first
 * step until mot_reset). w_out (nullable) receives w_i as [B][2][ne];
 * host or device memory (detected). stream: a cudaStream_t or NULL for the
 * default stream. Errors: MOT_ENOCONV (GMRES/CG limit hit; w_i is the last
 * iterate and the step counts), MOT_EINVAL, MOT_ESTATE, MOT_ECUDA.
 */
int mot_step(mot_handle* h, const mot_wave* waves, int B, double* w_out, void* stream);

/* n_steps calls of mot_step; w_out (nullable) receives [n_steps][B][2][ne]. */
int mot_run(mot_handle* h, int n_steps, const mot_wave* waves, int B, double* w_out, void* stream);

/*
 * March n scatterers of uneven sizes n_steps each, concurrently. The paper
 * marches one scatterer at a time (Section V-A, Eq. (MOT)); the scatterers
 * here are independent problems, each the same march. Scatterer i is marched
 * as by
 *   mot_run(hs[i], n_steps, waves[i], B[i], w_out ? w_out[i] : NULL, .)
 * on a stream of its own driven by a host thread of its own: each stream
 * starts after the work already queued on `stream` and `stream` waits for all
 * of them before its later work, so the latency-bound solves of the small
 * scatterers overlap the kernels of the large ones. The scatterers on the
 * tensor-core history (mixed precision, B a multiple of 8; up to 32, of the
 * first one's kernel form) march in lock step: every step, their history
 * contractions run as ONE launch of the history kernel over all of them (each
 * CTA serving one chunk of one scatterer), the rest of each step on its own
 * stream; that group is tuned once (mot_tune) at the first step that
 * contracts every member's full history. A scatterer outside the group gives
 * the results of the single mot_run (same kernels, same order); one inside it
 * those of a single march with the same tuned configuration (the history sums
 * of a chunking differ from another's by rounding).
 *   hs      : n distinct handles with operators loaded, on the device of
 *             `stream` (a cudaStream_t, or NULL for the default stream).
 *   waves   : n arrays, waves[i] holding B[i] plane waves (host).
 *   B       : n batch sizes, each in [1, 64] (fixed per handle as in mot_step).
 *   w_out   : NULL, or n pointers, each NULL or [n_steps][B[i]][2][ne_i]
 *             doubles in host or device memory.
 * Returns MOT_OK; MOT_ENOCONV if a step of some scatterer hit an iteration
 * limit; otherwise the error of the lowest-indexed scatterer that failed (its
 * message in that handle's mot_last_error; the others still finish). Errors
 * found before any work: MOT_EINVAL (n < 0, n_steps < 0, a NULL or repeated
 * handle, NULL waves or B). n == 0 returns MOT_OK.
 */
int mot_run_many(mot_handle* const* hs, int n, int n_steps, const mot_wave* const* waves, const int* B,
                 double* const* w_out, void* stream);

/*
 * Autotuner of the tensor-core history contraction (the paper has no
 * counterpart; it only picks how the work of Eq. (MOT)'s history sum is cut).
 * For n handles marched together (n = 1: one handle alone; n <= 32), every
 * candidate configuration -- tasks per chunk in {256, 512, 1024}, fraction of
 * the L2 a lag range may fill in {0.2, 0.4, 0.8}, pipeline stages x tasks
 * per stage in {4 x 1, 5 x 1, 2 x 2, 3 x 2} where they fit in shared memory,
 * epilogue warps in {4, 8} -- is applied and its launch (one
 * for all n handles) timed
 * three times with CUDA events on `stream` after one warm-up; the fastest
 * (median) is kept by every handle and reported by mot_get_info. The trial
 * launches read the current march state and change nothing a later step
 * reads. Requires handles on the tensor-core history (mixed precision, B a
 * multiple of 8) of one kernel form on one device that have taken a step
 * (MOT_ESTATE otherwise). mot_run_many tunes its group by itself, once, at
 * the first step that contracts every member's full history.
 */
int mot_tune(mot_handle* const* hs, int n, void* stream);

/*
 * Applies one configuration of the tensor-core history contraction without
 * timing any (e.g. one mot_tune chose for the same mesh and batch before):
 * tasks per chunk cap in [1, 1024], lag_frac in (0, 1], (stages,
 * tasks_per_stage) one of (4, 1), (5, 1), (2, 2), (3, 2), epilogue_warps 4
 * or 8. Only how the work of Eq. (MOT)'s history sum is cut changes; every
 * configuration computes the same sums. Same requirements as mot_tune
 * (MOT_ESTATE otherwise); MOT_EINVAL for a value out of range or a
 * configuration whose pipeline does not fit in shared memory (the handle's
 * previous configuration is then replaced by the chunking of cap and
 * lag_frac with its old pipeline). mot_get_info reports it with tc_tuned 0.
 */
int mot_set_tc_config(mot_handle* h, int cap, double lag_frac, int stages, int tasks_per_stage, int epilogue_warps);

/* Recovered currents of the last step, [B][4][ne]: j loop, j star, m loop,
 * m star (Eq. (dis_jm)), host or device memory. Ordered after the handle's
 * last mot_step, whatever stream that step ran on. */
int mot_get_currents(mot_handle* h, double* out);

/*
 * Scattered far field (after stepping) in the exterior medium, normalised by
 * the incident pulse spectrum at the origin, for every frequency set with
 * mot_set_frequencies and every unit direction dirs[n_dir][3] (host):
 *   E_inf(r) = (j k / 4 pi) [eta r x (r x N) + r x L],
 *   N = int J^(y) e^{j k r.y}, L = int M^(y) e^{j k r.y},
 * J^, M^ the exact Fourier transforms of the piecewise-constant currents.
 * E_out (host): [B][n_freq][n_dir][3] complex as (re, im) pairs. Ordered
 * after the handle's last mot_step, whatever stream that step ran on.
 */
int mot_fields(mot_handle* h, const mot_wave* waves, int n_dir, const double* dirs, double* E_out);

/*
 * mot_fields_noalloc: the same far field as mot_fields, computed without
 * allocating device memory during the call. The paper has no counterpart; it
 * exists for callers that may not call cudaMalloc / cudaFree at that point,
 * e.g. an application whose memory pool owns all device memory after start-up,
 * or a latency-critical loop in which allocation would synchronise the device.
 * mot_fields allocates staging buffers for the directions and the result on
 * every call; this variant stages them in one fixed device array of 262144
 * doubles (2 MiB) built into the library, which every GPU that loads the
 * library keeps until the process exits.
 *   Limit: 3*n_dir + 6*B*n_freq*n_dir <= 262144, else MOT_EINVAL with a message.
 *   The first call on a device looks up the array's device address (once per
 *   device); make that first call before any stream capture. The address is
 *   kept for the life of the process: a device reset between calls is not
 *   supported.
 *   All calls share the array: calls whose GPU work overlaps race on it, so the
 *   caller must serialise them. Arguments and E_out layout as for mot_fields.
 */
int mot_fields_noalloc(mot_handle* h, const mot_wave* waves, int n_dir, const double* dirs, double* E_out);

/* Restart the march at step 0 (operators kept). */
int mot_reset(mot_handle* h);

/* Save / restore the march state (step index, history ring, Fourier sums).
 * mot_save_state with buf == NULL returns the size in *size. */
int mot_save_state(mot_handle* h, void* buf, size_t* size);
int mot_load_state(mot_handle* h, const void* buf, size_t size);

int mot_get_info(mot_handle* h, mot_info* info);

/* Canonical edge table built by mot_create: ev[ne][2] (v^-, v^+),
 * ef[ne][2] (c^+, c^-) (host output arrays). */
int mot_get_edges(mot_handle* h, int32_t* ev, int32_t* ef);

const char* mot_last_error(mot_handle* h);

void mot_destroy(mot_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* MOT_H */
