// Internal declarations of the GB300 MOT library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include <string>
#include <vector>

#include "../../include/mot.h"

// Edge-block size of the block-sparse history tiles (rows and columns).
#define MOT_TILE 32
// Largest batch of plane waves per handle.
#define MOT_MAX_B 64
// Tasks per CTA of the tensor-core history kernel (staged in shared memory).
#define MOT_TC_CHUNK 1024
// Scatterers one launch of the tensor-core history kernel serves at most.
#define MOT_TC_MAX_JOBS 32
// Size (doubles) of the fixed device array used by mot_fields_noalloc.
#define MOT_NOALLOC_FIELD_DOUBLES 262144

// One tile product of the history contraction:
//   out[code.out] (TILE rows of row block rb, 2B columns)
//     += tile (TILE x TILE) * panel(k, code.part, code.variant)[rows of column block cb]
// part: 0 = loop coefficients l_{i-k}, 1 = star coefficients s_{i-k},
//       2 = windowed sum W_k of l (constant tail of K~).
// variant: 0 = [eta u, v / eta], 1 = [eta' u, v / eta'], 2 = [-v, u].
struct HistTask {
    int tile;
    int cb;
    int k;
    int code;  // part | variant << 2 | out << 4
};

struct HistChunk {
    int rb;
    int first;
    int count;
};

// Fixed FP64 matrix prepared for the emulated FP64 products on tensor cores:
// six bf16 integer slices per value (rows scaled by 2^-ea), pre-arranged in
// the MMA's layout, [Mp / 128][K / 32][6][128 x 32].
struct EmuMat {
    int M = 0, K = 0, Mp = 0, nsl = 6;  // slices per value: 6 (FP64-accurate) or 4 (beyond FP32)
    int* ea = nullptr;        // [Mp] row exponents
    uint16_t* a16 = nullptr;  // slices
};

// Device CSR matrix.
struct DCsr {
    int n = 0, m = 0;
    int64_t nnz = 0;
    int* rowptr = nullptr;
    int* col = nullptr;
    double* val = nullptr;
};

// Task list of one block-sparse contraction (history lags, or lag 0 inside Q_0).
struct TaskList {
    HistTask* tasks = nullptr;
    HistChunk* chunks = nullptr;
    int ntasks = 0;
    int nchunks = 0;
    int* chunk_ptr = nullptr;  // [nrb+1] chunk range of each row block (device)
    // lists whose chunks of one row block are not contiguous: the chunks of
    // row block rb are rb_chunks[rb_ptr[rb] .. rb_ptr[rb+1]) (device)
    int* rb_ptr = nullptr;
    int* rb_chunks = nullptr;
    // tensor-core list: merged tasks, x = tile for s1, y = tile for s2 (the
    // zero tile if absent), z = cb | k << 16 | (part | variant << 2) << 26
    uint4* packed = nullptr;
    int cap = 0;  // tensor-core list: most tasks in one chunk (staged in shared memory)
};

struct mot_handle {
    std::string err;
    int dev = 0;
    mot_options opt{};
    // geometry and material
    int nv = 0, nf = 0, ne = 0, npad = 0, nrb = 0;
    double eps_r = 1, mu_r = 1, dt = 0, D = 0, tmax = 0, c = 1, cp = 1, eta = 1, etap = 1;
    int kmax = 0, K = 0, R = 0;
    std::vector<double> verts;
    std::vector<int> tris, ev, ef, eo;
    std::vector<int> perm, iperm;  // perm[p] = canonical edge at internal row p
    bool loaded = false;

    // topology on device (internal edge order)
    int* d_edge_faces = nullptr;   // [ne][2] c+, c-
    int* d_edge_verts = nullptr;   // [ne][2] v-, v+
    int* d_face_edges = nullptr;   // [nf][3] internal edge ids
    double* d_face_sgn = nullptr;  // [nf][3]
    DCsr vtx_edges;                // vertex -> edges with sign (Lambda^T)
    DCsr Lf, Lv;                   // Sigma^T Sigma (faces), Lambda^T Lambda (vertices)
    DCsr G, Gt;                    // Gram matrix and its transpose (internal order)
    double* d_T0s = nullptr;       // [npad][npad]
    double* d_T0h = nullptr;
    int nq = 0;
    double* d_rhs_x = nullptr;     // [npad][nq][3]
    double* d_rhs_wf = nullptr;

    // block-sparse history
    double* d_tiles = nullptr;     // FP64 tiles (mixed path: lag 0 only, compact numbering, until set-up ends)
    int64_t ntiles = 0;
    int64_t ntiles_fp64 = 0;       // tiles held in FP64 (all; on the mixed path only those of lag 0)
    double tile_fill = 0;
    TaskList hist, lag0;
    TaskList hist_tc_list;  // tensor-core history: chunks = (lag range, row block) pieces, lag range major
    int max_tail_lag = 0;  // windows W_a needed for a in [1, max_tail_lag]

    // march state (allocated at the first step for a batch size B)
    int B = 0;
    int64_t step = 0;
    double* d_waves = nullptr;     // [B][10]
    std::vector<double> h_waves;
    double* d_ring = nullptr;      // [R][2 parts][3 variants][npad][2B]
    double* d_win = nullptr;       // [max_tail_lag+1][npad][2B]
    double* d_cur = nullptr;       // [4][npad][B] recovered currents of the last step
    double* d_wprev1 = nullptr;    // w_{i-1}, w_{i-2} (internal layout): GMRES initial guess
    double* d_wprev2 = nullptr;
    int* d_colidx = nullptr;       // [nrb][npad] column order of each row block (distance sorted)
    int nfreq = 0;
    std::vector<double> omega;
    double* d_omega = nullptr;
    double* d_dft = nullptr;       // [nfreq][4][npad][B][2]
    // work buffers
    double* d_work = nullptr;
    size_t work_bytes = 0;
    double* d_partial = nullptr;   // [nchunks][2][TILE][2B]
    size_t partial_bytes = 0;
    // GMRES
    int gm_m = 0;
    double* d_V = nullptr;         // [(m+1)][npad][2B]
    double* d_H = nullptr;         // [B][m+1][m]
    double* d_g = nullptr;         // [B][m+1]
    double* d_cs = nullptr;
    double* d_sn = nullptr;
    double* d_hcol = nullptr;      // [2][m+1][B] CGS2 coefficients
    double* d_red = nullptr;       // reduction scratch
    size_t red_bytes = 0;
    double* d_resid = nullptr;     // [B]
    double* h_resid = nullptr;     // pinned [B]
    int* d_iperm = nullptr;        // [ne] canonical edge -> internal row
    int* d_gm_active = nullptr;    // [B] GMRES system still iterating
    int* d_gm_jend = nullptr;      // [B] Krylov dimension reached
    double* d_gm_bnorm = nullptr;  // [B] |b|
    double* d_wscale = nullptr;    // [B] power-of-two scale of each wave's Q_0 system in the step
    int* d_cg_iters = nullptr;     // [0] max CG iterations, [1] non-converged solves,
                                   // [2] tensor-core history: code of a wait that ran out (0 = none)
    int* h_cg_iters = nullptr;     // pinned
    int last_gmres_iters = 0;
    int64_t gmres_iters_total = 0;  // since the march (re)started
    double last_gmres_resid = 0;
    int last_cg_iters = 0;
    int64_t launches = 0;
    int64_t device_bytes = 0;
    cudaStream_t stream = nullptr;
    // algorithmic work of a full-depth history contraction
    double hist_nnz_tasks = 0;   // sum over history tasks of the tile's nonzeros
    double hist_nnz_unique = 0;  // nonzeros of the stored tiles used by the history list
    // mixed-precision path (MOT_PREC_MIXED)
    float* d_tiles32 = nullptr;    // FP32 copy of the history tiles
    uint16_t* d_tiles16 = nullptr; // tensor-core path: the tiles as three bf16 slices in the MMA's B layout
    float* d_ring32 = nullptr;     // FP32 copy of the coefficient ring
    float* d_win32 = nullptr;      // FP32 windowed sums
    uint16_t* d_ring16 = nullptr;  // tensor-core path: bf16 slices of l and s, [R][2 parts][3 slices][npad][2B]
                                   // (bulk form: [npad x 128] per slice, in swizzled 32-row blocks)
    uint16_t* d_win16 = nullptr;   // tensor-core path: bf16 slices of the windowed sums, [a][3 slices][npad][2B]
    bool tc_bulk = false;          // tensor-core history in the bulk form (global column order, blocked ring)
    int tc_stages = 0;             // pipeline stages of the tensor-core history (0: the deepest that fits)
    int tc_cap = 0;                // tasks per chunk the tensor-core list was cut with
    int tc_epi = 4;                // epilogue warps of the tensor-core history (4 or 8)
    int tc_tps = 1;                // tasks per pipeline stage of the tensor-core history (1 or 2)
    // FP64 path with fp64_direct: dense inverses formed at load, in place of CG
    double* d_Ginv64 = nullptr;    // G^{-1}, npad x npad
    double* d_Lfinv64 = nullptr;   // (L_f + 11^T/N_f)^{-1}, dfpd x dfpd (identity on the padding)
    double* d_Lvinv64 = nullptr;   // (L_v + 11^T/N_v)^{-1}, dvpd x dvpd
    int dfpd = 0, dvpd = 0;
    double* d_dir_r = nullptr;     // direct Laplacian solves: right-hand side and solution,
    double* d_dir_z = nullptr;     // max(dfpd, dvpd) x 4 MOT_MAX_B each, and column scales
    double* d_dir_sc = nullptr;
    double tc_lag_frac = 0;        // fraction of L2 a lag range of the list may fill
    bool tc_tuned = false;         // the three were chosen by mot_tune
    float tc_tune_ms = 0;          // the chosen configuration's launch time in the tuning (ms)
    int64_t tc_launches = 0;       // history-kernel launches that served this handle
    std::vector<HistTask> tc_tasks_host;  // the tensor-core list's tasks (host), for re-chunking
    std::vector<int> tc_rbs_host;
    bool hist_tc = false;          // history contraction on the tensor cores (mixed path, B a multiple of 8)
    double* d_Q0 = nullptr;        // dense Q_0, (2 npad)^2, interleaved (edge, component) order, FP64
    float* d_Q0f = nullptr;        // FP32 copy
    double* d_LF = nullptr;        // dense [M1 | M2], npad x 2 npad, FP64
    float* d_LFf = nullptr;        // FP32 copy
    float* d_xf = nullptr;         // FP32 staging: [2 bv]
    double* d_sgws = nullptr;      // split-K partial results of the FP32 dense products
    size_t sgws_bytes = 0;
    EmuMat emu_Q0, emu_LF;         // Q_0 and [M1 | M2] for the emulated FP64 products (MOT_MIX_EMU64)
    EmuMat emu_Q0s, emu_Minv;      // Q_0 and Q_0^{-1} with 4 slices: the products of the FP32 solves
    unsigned char* d_emuws = nullptr;  // their per-call workspace (X slices, split-K partials)
    size_t emuws_bytes = 0;
    float* d_Minvf = nullptr;      // FP32 Q_0^{-1} (GMRES preconditioner), (2 npad)^2
    double* d_Minv64 = nullptr;    // FP64 Q_0^{-1} (preconditioner of the FP64 path, fp64_precond)
    bool prec_active = false;      // apply_q0 computes Q_0 M v
    float* d_Lfinvf = nullptr;     // FP32 (Sigma^T Sigma + 11^T/N_f)^{-1}, nfpd x nfpd (CG preconditioner)
    int nfpd = 0;                  // N_f padded to 64
    double* d_pcg_work = nullptr;  // 5 x nfpd x 2B
    double* d_pcg_scal = nullptr;  // 6 x 2B doubles + 2B ints
    float* d_pcg_f32 = nullptr;    // nfpd x 2B
    int last_pcg_iters = 0;
    bool precomputing = false;     // dense operators being assembled (use the product form)
    double gm_tol = 1e-12;         // relative tolerance of the GMRES solve in progress
    int refine_sweeps = 0;         // FP64 refinement sweeps used by the last step
    // CUDA-event timing of the history launches (mot_options.timing)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // recorded on the stepping stream at the end of every mot_step: the calls
    // that read the march state on the legacy stream (currents, far field)
    // wait for it, whatever stream the handle last stepped on
    cudaEvent_t ev_state = nullptr;
    cudaEvent_t pev[8] = {nullptr};  // step phase boundaries
    double phase_ms[8] = {0};
    bool ev_pending = false;
    int64_t timed_launches = 0;
    double timed_ms = 0;
};

// ---- kernels' host wrappers (implemented in the .cu files) ----
namespace mot {

// error helpers
int fail(mot_handle* h, int code, const std::string& msg);

// Runs f (an idempotent per-device setting, e.g. a kernel's shared-memory
// attribute) the first time a call site reaches it on device dev; safe when
// several host threads reach it at once (f may then run more than once).
template <class F>
inline void once_per_device(std::atomic<unsigned long long>& done, int dev, F&& f) {
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    f();
    done.fetch_or(bit, std::memory_order_acq_rel);
}
int cuda_fail(mot_handle* h, cudaError_t e, const char* where);
void* dalloc(mot_handle* h, size_t bytes);

// history
void launch_history(mot_handle* h, const TaskList& tl, const double* tiles, const double* ring, const double* win,
                    const double* kry, int mode, long long step_i, double* out_s1, double* out_s2, cudaStream_t s);

// tensor-core history (mixed path, B a multiple of 8): tiles from d_tiles16, panels from d_ring16/d_win16
void launch_history_tc(mot_handle* h, const TaskList& tl, long long step_i, double* out_s1, double* out_s2,
                       cudaStream_t s);
// sum of the chunk partial results of a history launch into out_s1 / out_s2
void launch_history_reduce(mot_handle* h, const TaskList& tl, int C2, double* out_s1, double* out_s2,
                           cudaStream_t s);
// npanels FP64 panels of npad x 2B values -> three bf16 slices each
void launch_split3(mot_handle* h, int npanels, const double* src, uint16_t* dst, cudaStream_t s);
// bf16 slices of the FP32 tiles in the tensor core's B layout (d_tiles32 -> d_tiles16)
void launch_split_tiles(mot_handle* h, cudaStream_t s);
// bf16 slices of l and s of ring slot `slot` (from the FP64 ring's [-v, u] variant)
void launch_split_ring(mot_handle* h, int slot, cudaStream_t s);
bool history_tc_fits(int npad, bool bulk);  // the kernel's shared memory fits (gathered form: with the column order)
size_t history_tc_ring_slot_elems(const mot_handle* h);  // bf16 elements of one ring slot of d_ring16
int history_tc_stages(int npad, bool bulk, int cap);
// whether (ns stages of tp tasks) fits the kernel's shared memory with cap staged tasks
bool history_tc_config_fits(int npad, bool bulk, int cap, int ns, int tp);
float launch_history_tc_many(mot_handle* const* hs, int n, double* const* s1, double* const* s2, cudaStream_t s,
                             bool timed);

// emulated FP64 products on tensor cores (k_emu64.cu): Y (M x N) = A X with A
// prepared once by emu_prepare from the device FP64 matrix A (M x K, ld K)
int emu_prepare(mot_handle* h, const double* A, int M, int K, EmuMat* out, int nsl);
void emu_free(mot_handle* h, EmuMat* m);
int launch_emu_gemm(mot_handle* h, const EmuMat& A, const double* X, int N, double* Y, cudaStream_t s);

// block-vector helpers (rows npad, C columns)
void launch_axpby(mot_handle* h, int n, double a, const double* x, double b, const double* y, double* z,
                  cudaStream_t s);  // z = a x + b y, n doubles
void launch_variants(mot_handle* h, const double* x, double* dst, double eta, double etap, cudaStream_t s);
void launch_sigma_t(mot_handle* h, const double* x, int C, double* f, cudaStream_t s);   // faces <- edges
void launch_sigma(mot_handle* h, const double* z, int C, double* x, cudaStream_t s);     // edges <- faces
void launch_lambda_t(mot_handle* h, const double* x, int C, double* v, cudaStream_t s);  // vertices <- edges
void launch_lambda(mot_handle* h, const double* z, int C, double* x, cudaStream_t s);    // edges <- vertices
void launch_spmv(mot_handle* h, const DCsr& A, const double* x, int C, double* y, cudaStream_t s);
int launch_cg(mot_handle* h, const DCsr& A, const DCsr* A2, const double* f, int C, double* z, double* work,
              cudaStream_t s);  // returns max iterations or -1 on no convergence
void launch_gemm(mot_handle* h, const double* A, const double* X, int C, double* Y, cudaStream_t s);
// Y[M][C] = A[M][K] X[K][C], FP64
void launch_gemm_rect(mot_handle* h, int M, int K, const double* A, const double* X, int C, double* Y,
                      cudaStream_t s);
void launch_rhs(mot_handle* h, long long i, double* rho1, double* rho2, cudaStream_t s);
void launch_window_sums(mot_handle* h, long long i, cudaStream_t s);
void launch_recover(mot_handle* h, long long i, cudaStream_t s);
void launch_pack_w(mot_handle* h, const double* x, double* out, cudaStream_t s);  // internal -> [B][2][ne]

// GMRES pieces
void launch_gm_dots(mot_handle* h, const double* V, int nvec, const double* w, double* out, cudaStream_t s);
void launch_gm_update(mot_handle* h, const double* V, int nvec, const double* coef, double* w, cudaStream_t s);
void launch_gm_norm(mot_handle* h, const double* w, double* out, cudaStream_t s);
void launch_gm_scale(mot_handle* h, const double* w, const double* nrm, double* v, cudaStream_t s);
void launch_gm_arnoldi_finish(mot_handle* h, int j, const double* hcol, const double* nrm, cudaStream_t s);
void launch_gm_init(mot_handle* h, const double* beta, int first_cycle, cudaStream_t s);
// power-of-two scale of every wave's system (sc[b] = 2^-e) and its application
void launch_wave_scale(mot_handle* h, const double* x, double* sc, cudaStream_t s);
void launch_wave_apply(mot_handle* h, const double* sc, bool inverse, double* x, cudaStream_t s);
void launch_gm_solve_update(mot_handle* h, double* y, double* x, cudaStream_t s);

}  // namespace mot
