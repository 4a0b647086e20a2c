// rw_internal.h -- host-side structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rw_common.cuh"
#include "rwpc.h"

struct rw_context {
    cudaStream_t stream = nullptr;
    rw_alloc_fn alloc = nullptr;
    rw_free_fn free_fn = nullptr;
    void* user = nullptr;
    rw_options opt{};
    int device = 0;
    int num_sms = 0;
    rw::DevStatus* d_status = nullptr;  // device copy
    rw::DevStatus* h_status = nullptr;  // pinned host copy
    void* h_small = nullptr;            // pinned host scratch (256 bytes)
    double reuse_ratio = 8.0;           // walk reuse: extra records per walk to allocate for
    size_t l2_bytes = 0;                // L2 cache size of the device
    cudaEvent_t ev[16] = {};
};

namespace rw {

// NVTX range over a host scope: a profiler attributes the kernels launched
// inside it to that phase of the library (for example
// ncu --nvtx --nvtx-include "rw_walk/").  Without a profiler attached the
// calls return at once.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kFeatures = RW_NUM_FEATURES;
constexpr int kFeatStride = RW_FEATURE_STRIDE;
constexpr int kMlpParams = RW_MLP_PARAMS;

void set_error(const char* fmt, ...);

// Kernels launched by the calling thread (reported per call in the factor
// description and the PCG statistics).
extern thread_local int64_t g_launches;
#define RW_COUNT_LAUNCH() (++rw::g_launches)

// Device allocations made through the context's allocator.
struct Pool {
    rw_context* ctx = nullptr;
    struct Buf {
        void* p;
        size_t bytes;
    };
    std::vector<Buf> bufs;
    explicit Pool(rw_context* c = nullptr) : ctx(c) {}
    void* get(size_t bytes);   // nullptr on failure (error message set)
    void release(void* p);     // free one allocation now
    void release_all();
    ~Pool() { release_all(); }
    Pool(const Pool&) = delete;
    Pool& operator=(const Pool&) = delete;
};

template <typename T>
inline T* alloc_n(Pool& pool, int64_t n) {
    return static_cast<T*>(pool.get(sizeof(T) * (size_t)(n > 0 ? n : 1)));
}

// Exclusive prefix sum of n values; out has n + 1 entries (out[n] = total).
// Works for in == out.  tmp: scratch from the pool.
cudaError_t scan_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s, Pool& pool);
cudaError_t scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n, cudaStream_t s,
                            Pool& pool);
cudaError_t scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, Pool& pool);

inline int grid_for(int64_t work, int block, int max_blocks) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

// ---- build path (rw_tables.cu, rw_walk.cu, rw_emit.cu, rw_levels.cu) -------

// Walk tables of one matrix, in the layout read by the walk kernel.
//  tab:   32-byte sectors of 8 uint32 words in four regions.  A node's slots
//         (slot 0 = header, slot s + 1 = successor s in ascending column
//         order) form ng = ceil((1 + deg) / 4) groups; slot j lives in group
//         j / 4, word j % 4 its threshold (0 for the header slot: always
//         passed), word 4 + j % 4 its successor word (the successor's node
//         index in bits 27..0, in bits 31..28 its class: 0 without a
//         summary, ng for 3 <= ng <= 8, 15 above; deg for the header slot,
//         0 for padding).
//           sectors [0, 2n): node j's groups at 2j, 2j + 1 when ng <= 2;
//           sectors [2n, 3n): node j's summary at 2n + j when ng > 2 -- deg in
//             word 0, in words 1..7 the last threshold of groups 0..6
//             (0xFFFFFFFF past the last);
//           sectors [3n, 11n): node j's groups at 3n + 8j when 2 < ng <= 8
//             (a fixed stride, so that a group's address needs no load);
//           sectors [11n, 11n + G): the groups of the nodes with more than
//             eight, at gbase[j] (a prefix over those nodes).
//         The summaries (32 bytes per node, dense) stay in L2 on large
//         matrices, so a hop to a node with a summary costs one DRAM sector
//         (its group) besides one L2 read (two, with gbase, above eight
//         groups); a node of at most seven neighbours costs one or two
//         sectors of group 0/1.  Sectors [3n, 11n) are allocated for every
//         node but touched only by the nodes that use it.
//  gbase: [n] the sector of each node's group 0.
//  fthr:  per walk row a block [updeg, lowdeg, ft_0 .. ft_{updeg-1}, pad].
// The walk works with node indices throughout (home: below the start row,
// return: equal to it).  Padding thresholds are 0xFFFFFFFF.
struct Tables {
    int32_t n = 0;
    uint32_t* tab = nullptr;
    uint32_t* gbase = nullptr;    // [n] sector of each node's group 0
    uint32_t* fthr = nullptr;
    uint32_t* toff = nullptr;     // [n+1] groups of the nodes with more than eight groups before each node
    uint32_t* foff8 = nullptr;    // [n+1] first-step blocks (32-byte blocks)
    int32_t* deg = nullptr;       // [n] off-diagonal count
    int32_t* lowdeg = nullptr;    // [n] entries with column < row
    double* S = nullptr;          // [n] sum_{j>k} A_kj
    double* diag = nullptr;       // [n] A_kk
    int32_t* diag_pos = nullptr;  // [n] CSR position of the diagonal
    uint32_t* walk_flag = nullptr;    // [n+1] scanned into the walk-row index
    int32_t n_walk_rows = 0;
    int4* wrow = nullptr;         // [n_walk_rows] {k, foff8_k, gbase_k, lowdeg_k}
    int32_t* walk_rows = nullptr; // [n_walk_rows] k ascending
    uint64_t sectors = 0, first_words = 0;
};

rw_status build_tables(rw_context* ctx, const rw_csr* A, Tables& T, Pool& pool);

// Per-walk-row budgets and the walk index space.
struct WalkSpace {
    int64_t total = 0;            // total walks
    int64_t* wbase = nullptr;     // [n_walk_rows + 1]
    int32_t* chunk_row = nullptr; // [nchunks]
    int64_t nchunks = 0;
};
constexpr int kWalkChunk = 32;

rw_status build_walk_space(rw_context* ctx, const Tables& T, uint32_t uniform,
                           const uint32_t* d_budget, WalkSpace& ws, Pool& pool, bool allow_zero = false);
// chunk_row[c] = the walk row holding walk c * kWalkChunk (wbase: [nw+1]).
rw_status build_chunk_rows(rw_context* ctx, int32_t nw, const int64_t* wbase, int32_t* chunk_row);

struct WalkLaunch {
    uint64_t max_steps = 1ull << 24;
    int record_lengths = 0;
};

// Tables, key and tag of one matrix as the walk kernel reads them.  The tag
// is (matrix_index << 2) | kind (kind 0: factor walks, 1: pilot walks).
struct MatWalk {
    const uint32_t* tab;
    const uint32_t* gbase;
    const uint32_t* fthr;
    uint32_t key0, key1, tag, n;  // n: nodes (the summaries start at sector 2n)
};

// The walk index space of one launch (one matrix, or several concatenated).
struct WalkBatch {
    int nmat = 1;
    uint64_t table_bytes = 0;      // walk-table bytes of all matrices
    int32_t nrows = 0;             // walk rows of all matrices
    MatWalk m0{};                  // the single matrix (nmat == 1)
    const MatWalk* mats = nullptr; // [nmat] device (nmat > 1)
    const int32_t* wmat = nullptr; // [walk rows] matrix of each walk row (nmat > 1)
    const int4* wrow = nullptr;
    const int64_t* wbase = nullptr;
    const uint32_t* wofs = nullptr;  // first walk index of each walk row (NULL: 0)
    const int32_t* chunk_row = nullptr;
    int64_t total = 0;
};

inline uint64_t table_bytes(const Tables& T) { return T.sectors * 32u + (uint64_t)T.n * 4u; }

inline MatWalk mat_walk(const Tables& T, uint64_t seed, uint32_t matrix_index, uint32_t kind) {
    return MatWalk{T.tab, T.gbase, T.fthr, (uint32_t)seed, (uint32_t)(seed >> 32),
                   (matrix_index << 2) | (kind & 3u), (uint32_t)T.n};
}

rw_status run_walks(rw_context* ctx, const WalkBatch& wb, const WalkLaunch& wl, int2* rec,
                    unsigned long long* d_hops, Pool& pool, float* ms);

// Sub-walks extracted by walk reuse (Algorithm 2), bucketed per walk row:
// row r's records {end node or -1, returns} are xrec[xbase[r] .. xbase[r+1]).
struct Extras {
    int64_t count = 0;
    int64_t* xbase = nullptr;  // [n_walk_rows + 1]
    int2* xrec = nullptr;      // [count]
    int32_t* xnode = nullptr;  // unbucketed: start node, end, returns
    int32_t* xend = nullptr;
    uint32_t* xret = nullptr;
};

// The walks of a single-matrix launch with reuse: rec as run_walks, and the
// extracted sub-walks in X (allocated from xpool, which must outlive the merge).
rw_status run_walks_reuse(rw_context* ctx, const WalkBatch& wb, const WalkLaunch& wl, const Tables& T, int2* rec,
                          unsigned long long* d_hops, Pool& pool, Pool& xpool, float* ms, Extras& X);

// Merge + emission: per-walk records -> Y (CSR), D, counters.
struct FactorOut {
    int64_t nnz = 0;
    int64_t* y_rp = nullptr;
    int32_t* y_col = nullptr;
    double* y_val = nullptr;
    double* d = nullptr;
    uint32_t* M = nullptr;
    uint64_t* J = nullptr;
    uint32_t* G = nullptr;
};

// X: the sub-walks of walk reuse (NULL without reuse); each counts as a walk
// of its start row.
rw_status emit_factor(rw_context* ctx, const rw_csr* A, const Tables& T, const WalkSpace& ws,
                      const int2* rec, const Extras* X, double drop_tol, FactorOut& fo, Pool& pool,
                      Pool& scratch, float* ms_merge, float* ms_emit);

// Stable LSD radix sort (9-bit digits) of cnt (key, value) pairs on the low
// `bits` bits of the keys, ping-ponging between (k0, v0) and (k1, v1); *ko, *vo
// receive the pair of buffers that holds the result.
rw_status radix_sort_pairs(rw_context* ctx, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t cnt,
                           int bits, Pool& scratch, uint32_t** ko, uint32_t** vo);

rw_status transpose_factor(rw_context* ctx, int32_t n, const FactorOut& fo, int64_t* yt_rp,
                           int32_t* yt_col, double* yt_val, Pool& scratch);

// Level order of a triangular solve: rows sorted by level of the dependency
// DAG of the strict triangular CSR (rp, col); descending = upper triangular.
// *lptr_out (allocated from keep) receives the depth + 1 level boundaries.
struct LevelDag {
    const int64_t* rp;
    const int32_t* col;
    bool descending;
    int32_t* order;       // [n] out
    int32_t* depth;       // out
    int64_t** lptr_out;   // out
};
// The forward (Y) and backward (Y^T) DAGs in one launch.
rw_status compute_levels_pair(rw_context* ctx, int32_t n, const LevelDag& fwd, const LevelDag& bwd, Pool& keep,
                              Pool& scratch);

// Schedule of one triangular solve (see rw_sched.cu).
struct SolveRun {
    int thin;                    // 1: one block with shared-memory values; 0: whole grid
    int32_t lev_begin, lev_end;  // levels [begin, end)
    int64_t pos_begin, pos_end;  // positions in the level order
    int64_t in_entries = 0;      // thin run: entries whose column lies in the run
};
struct SolveSchedule {
    int32_t n = 0, depth = 0;
    const int32_t* order = nullptr;  // rows in level order
    const int64_t* lptr = nullptr;   // [depth + 1] level boundaries (device)
    std::vector<int64_t> lptr_h;     // host copy
    std::vector<SolveRun> runs;
    int64_t* tptr = nullptr;         // [n+1] packed entries of thin-run positions
    int32_t* tnin = nullptr;         // [n] in-run entries of each position (listed first)
    int32_t* tidx = nullptr;         // in-run: slot in the run; external: column
    double* tval = nullptr;
    float* tval32 = nullptr;
    int64_t thin_entries = 0;
};

rw_status build_schedule(rw_context* ctx, int32_t n, const int64_t* rp, const int32_t* col,
                         const double* val, const float* val32, const int32_t* order,
                         const int64_t* lptr_dev, int32_t depth, SolveSchedule& S, Pool& pool,
                         Pool& scratch);

// Device workspace of the solves, owned by the factor: two grid-barrier words
// (at offset 0) and the external sums of a thin run (from byte 256 on).
constexpr int64_t kSolveWorkspaceBytes = 256 + (int64_t)4096 * 16 * 8;

// w <- w / d row by row (w node-major [n][nrhs]), in place: the D^-1 step of
// the preconditioner between the two solves, so that the forward solve's rows
// need no division of their own (the FP64 division is a long instruction
// sequence on GB300's narrow FP64 pipe; here one instruction serves 32 rows).
// IEEE division as the solve would do it, so results are unchanged.
template <typename T>
rw_status apply_inverse_diag(rw_context* ctx, T* w, const T* d, int64_t n, int nrhs);

// backward: the Y^T solve (rw_options.solve_mode_bwd may choose its mode).
template <typename T>
rw_status solve_runs(rw_context* ctx, const SolveSchedule& S, const int64_t* rp, const int32_t* col,
                     const T* val, const T* tval, const T* rhs, const T* scale, T* x, int nrhs,
                     unsigned* bar, bool backward = false);

// ---- solve path (rw_solve.cu) ----------------------------------------------

struct FactorView {
    int32_t n;
    int64_t nnz;
    const int64_t* y_rp;
    const int32_t* y_col;
    const double* y_val;
    const float* y_val32;
    const int64_t* yt_rp;
    const int32_t* yt_col;
    const double* yt_val;
    const float* yt_val32;
    const double* d;
    const float* d32;
    const int32_t* fwd_order;
    const int32_t* bwd_order;
    const SolveSchedule* fwd_sched;
    const SolveSchedule* bwd_sched;
    unsigned* bar;  // grid-barrier words of the solves (owned by the factor)
};

void launch_to_fp32(const double* in, float* out, int64_t cnt, cudaStream_t s, int num_sms);
// FP32 operator of the mixed mode: off-diagonals rounded, the diagonal slot
// holding the row's excess e_i = A_ii + sum_j A_ij (applied by the FP32 SpMV as
// e_i x_i + sum_j A_ij (x_j - x_i)).
void launch_to_fp32_diff(int32_t n, const int32_t* rp, const int32_t* col, const double* val, float* a32,
                         cudaStream_t s, int num_sms);
rw_status spmv_fp64(rw_context* ctx, const rw_csr* A, const double* x, double* y, int nrhs);
rw_status precond_fp64(rw_context* ctx, const FactorView& F, const double* r, double* z,
                       int nrhs, Pool& scratch);
rw_status pcg_run(rw_context* ctx, const rw_csr* A, const FactorView& F, const double* b,
                  double* x, int nrhs, double tol, int max_iter, rw_precision prec,
                  rw_pcg_stats* stats, int32_t* h_iters, double* h_relres);
// BiCGSTAB (right preconditioning, one right-hand side, FP64) with the
// preconditioner of view F (see rw_solve.cu).
rw_status bicgstab_run(rw_context* ctx, const rw_csr* A, const FactorView& F, const double* b, double* x, double tol,
                       int max_iter, rw_pcg_stats* stats);
// B = A^T as a CSR with ascending columns (row_ptr [n+1], col and val [nnz]).
rw_status csr_transpose(rw_context* ctx, const rw_csr* A, int32_t* rp, int32_t* col, double* val, Pool& scratch);

// y = A x (node-major, nrhs <= 16) for T = double or float.
template <typename T>
rw_status spmv_launch(rw_context* ctx, int32_t n, const int32_t* rp, const int32_t* col, const T* val,
                      const T* x, T* y, int nrhs);

// Size and pointer checks of a matrix argument (RW_ERR_ARG / RW_ERR_NOT_RMATRIX).
rw_status check_csr(const rw_csr* A);

// What the schedule autotuner times: the SpMV operator and a factor with its
// solve schedules (a single factor or a batch).
struct TuneTarget {
    int32_t n;
    const int32_t* a_rp;
    const int32_t* a_col;
    const double* a_val;
    const float* a_val32;  // excess + difference form (may be NULL)
    const int64_t* y_rp;
    const int32_t* y_col;
    const double* y_val;
    const float* y_val32;
    const int64_t* yt_rp;
    const int32_t* yt_col;
    const double* yt_val;
    const float* yt_val32;
    const double* d;
    const float* d32;
    const SolveSchedule* fwd;
    const SolveSchedule* bwd;
    unsigned* bar;
    int64_t nnz_y;
    int32_t depth;
};
rw_status factor_tune_target(const rw_factor* F, const rw_csr* A, TuneTarget* X);

// Transpose, levels, FP32 copies and solve schedules of a factor whose rows
// are in fo (allocated from F->pool); fills F->desc's arrays.
rw_status complete_factor(rw_context* ctx, rw_factor* F, const FactorOut& fo, Pool& scratch);
rw_status batch_tune_target(const rw_batch* B, TuneTarget* X);

// Launch-and-check helper: returns RW_ERR_CUDA with a message on failure.
rw_status check_cuda(cudaError_t e, const char* what);
rw_status check_launch(const char* what);
// Kernel attributes (dynamic shared-memory limit, non-portable cluster sizes)
// belong to each device's context: set `attr` of `func` to `value` once per
// device (thread-safe; later calls on the same device return at once).
rw_status set_kernel_attr_once(int device, const void* func, cudaFuncAttribute attr, int value);
rw_status read_status(rw_context* ctx, const char* what);  // syncs, maps device flags
rw_status reset_status(rw_context* ctx);

}  // namespace rw

struct rw_factor {
    rw_context* ctx = nullptr;
    rw::Pool pool;
    rw_factor_desc desc{};
    int32_t* fwd_order = nullptr;
    int32_t* bwd_order = nullptr;
    rw::SolveSchedule fwd_sched, bwd_sched;
    unsigned* bar = nullptr;
    explicit rw_factor(rw_context* c) : ctx(c), pool(c) {}
};
