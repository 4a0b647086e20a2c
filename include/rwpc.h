/*
 * rwpc.h -- C ABI of the GB300 random-walk preconditioner library (librwpc.so).
 *
 * Method: H. Qian, S. S. Sapatnekar, "Stochastic Preconditioning for Iterative
 * Linear Equation Solvers".  For an R-matrix A (symmetric M-matrix, irreducibly
 * diagonally dominant, Sec. 1) the library runs the random-walk game of Sec. 2.1
 * (transition -A_ij/A_ii, absorption at the diagonal excess, Eq. map) with rows
 * 0..k-1 as homes for walks started at row k (Sec. 2.2.1), counts per start row
 * the journey record of Sec. 3.1 (walks M, end counts H, returns J), and turns
 * it into an incomplete factor with the one-step-exact estimator of Sec. 5.2
 * (Eqs. newy, newz) and a post-processing threshold drop (footnote of Sec. 4).
 * The factor is applied inside preconditioned conjugate gradients (Algorithm 1).
 *
 * Factor convention.  Indices are 0-based and in A's own order.  The library
 * returns Y (unit lower triangular; only the strict lower part is stored, CSR,
 * columns ascending) and D (diagonal) with  A ~= Y^T diag(D) Y.  In the paper's
 * notation this is L_rev(A) = rev(Y)^T and D_rev(A) = rev(D) (Eqs. y and d): the
 * paper's reversal is a relabelling only, so no data is reordered.
 *
 * Lifetime.  A factor allocates and frees through its context: destroy every
 * factor of a context before the context itself.
 *
 * Memory.  Every pointer inside rw_csr and every d_* argument is a DEVICE
 * pointer owned by the caller, on the device current when the context was made.
 * Factor storage and scratch are allocated by the library through the
 * context's allocator (cudaMallocAsync on the context stream by default) and
 * released by rw_factor_destroy / at the end of the call.  Host pointers are
 * marked h_*.
 *
 * Streams.  All device work of a call is enqueued on the context's stream.
 * Calls return after synchronising that stream whenever they return host data
 * (status, counts); device outputs are complete when the call returns.
 *
 * Errors.  Every entry point returns an rw_status (0 = RW_OK, negative =
 * error); no exception crosses the ABI.  rw_last_error() gives a message for
 * the last failing call of the calling thread.
 */
#ifndef RWPC_H
#define RWPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RW_OK = 0,
    RW_ERR_ARG = -1,            /* bad argument (null pointer, size, budget < 1, ...) */
    RW_ERR_NOT_RMATRIX = -2,    /* A is not in the required R-matrix form (see rw_csr) */
    RW_ERR_WALK_CAP = -3,       /* a walk reached rw_options.max_steps hops */
    RW_ERR_ALLOC = -4,          /* the allocator failed */
    RW_ERR_NO_CONVERGENCE = -5, /* PCG reached max_iter (tol > 0) */
    RW_ERR_BREAKDOWN = -6,      /* PCG found p.Ap <= 0 */
    RW_ERR_CUDA = -7,           /* a CUDA runtime call failed */
    RW_ERR_TIMEOUT = -8,        /* a bounded device-side wait gave up */
    RW_ERR_CAPACITY = -9        /* a fixed-size table is too small: a row has more than 2^29 possible
                                   end points (merge table limit), a matrix has 2^28 nodes or more or
                                   needs 2^31 walk-table sectors or more (the walk tables' index
                                   range), or n * nrhs exceeds the 2^20-entry scratch array of
                                   rw_precond_apply_static */
} rw_status;

typedef enum { RW_FP64 = 0, RW_FP32_MIXED = 1 } rw_precision;

/* Square CSR matrix on the device.  Requirements (checked, RW_ERR_NOT_RMATRIX):
 * row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz; columns strictly
 * ascending within a row and in [0, n); the diagonal is stored and positive;
 * every stored off-diagonal is strictly negative (no explicit zeros); every
 * row is diagonally dominant: A_ii + sum_{j != i} A_ij >= -1e-12 A_ii.
 * Symmetry and irreducibility are the caller's promise (not checked: a
 * component without ground makes walks run to the step cap, RW_ERR_WALK_CAP). */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int32_t* row_ptr; /* [n+1] */
    const int32_t* col;     /* [nnz] */
    const double* val;      /* [nnz] */
} rw_csr;

/* Optional allocator, e.g. a framework's caching allocator.  alloc returns a
 * device pointer aligned to 256 bytes or NULL; free releases it.  The stream
 * is the context stream (cudaStream_t passed as void*). */
typedef void* (*rw_alloc_fn)(void* user, size_t bytes, void* stream);
typedef void (*rw_free_fn)(void* user, void* ptr, size_t bytes, void* stream);

typedef struct {
    uint64_t max_steps;      /* walk step cap (default 1 << 24) */
    int32_t keep_records;    /* 1: keep the per-walk records in the factor (default 0) */
    int32_t record_lengths;  /* 1: records hold walk lengths instead of returns (default 0) */
    int32_t store_fp32;      /* 1: also keep FP32 copies of Y, Y^T and D (default 1) */
    int32_t refine_every;    /* FP32 PCG: true-residual replacement period (default 50) */
    int32_t walk_blocks_per_sm; /* 0 = from the occupancy calculator */
    int32_t timing;          /* 1: record per-phase device times (default 1) */
    int32_t solve_blocks_per_sm; /* wide-level solves and the sync-free parts with vector rows:
                                    512-thread blocks per SM (0 = 1; 2 = a register-capped
                                    sync-free kernel, two blocks resident per SM) */
    int32_t graphs;          /* 1: batched PCG replays each iteration from a CUDA graph (default 1) */
    int32_t wide_slices;     /* wide-level solves: entry slices per row (lanes per row = slices x
                                right-hand sides, power of two <= 32); 0 = one row per warp;
                                -1 = vector rows: one row per warp, each lane reads all
                                right-hand sides of its entries (default -1) */
    int32_t spmv_slices;     /* SpMV: entry slices per row, as wide_slices; 0 = one row per warp */
    int32_t cluster_width;   /* levels of at most this many rows (above the thin-run width) run on
                                one thread-block cluster with hardware barriers; 0 = never */
    int32_t cluster_size;    /* CTAs of that cluster (2..16; 0 = 16) */
    int32_t solve_mode;      /* triangular solves: 0 = level schedule (thin / wide / cluster runs),
                                1 = sync-free (each row waits only for its own dependencies),
                                2 = hybrid (thin runs on one block, the other runs sync-free;
                                default 2) */
    int32_t reuse;           /* 1: walk reuse (Algorithm 2 of Sec. 5.3) in single-matrix builds:
                                every simulated walk also counts, for each later node k' it
                                passes, the legal sub-walk from k' (k' its least node until it
                                ends below k' or at ground; one-step sub-walks excluded; walks of
                                one start row never overlap).  Y, D and the counters then hold
                                all these walks (default 0) */
    int32_t solve_mode_bwd;  /* solve_mode of the backward (Y^T) solve; -1 = as solve_mode (default) */
    int32_t thin_levels;     /* factor build: levels per thin run at most (0 = no cap; default 128);
                                dependencies on earlier runs are summed by the whole grid */
    int32_t thin_cluster;    /* thin runs on a thread-block cluster of this many CTAs (2..16, reduced to
                                what the device can place), x replicated in each CTA's shared memory;
                                0 or 1 = one block (default 0) */
    int32_t adapt_ahead;     /* rw_adaptive_budget: walks a row runs past its next decision point T, in
                                percent of T (default 100; 0 = exactly up to T); changes only the
                                time, never the counts */
    int32_t thin_flags;      /* thin runs on one block: 1 = each row flags its slot in shared memory
                                when done and readers wait on the flags of their entries (no barrier
                                per level); 0 = one block barrier per level (default 0) */
    int32_t spin_limit;      /* polls of one device-side wait (level computation, solve hand-offs,
                                grid and cluster barriers, the latency probe) before it gives up and
                                the call returns RW_ERR_TIMEOUT; 0 = 2^20 (about a second at L2
                                latency; default 0).  A small value makes waits give up early: for
                                testing the timeout path, never for results */
    int32_t thin_lanes;      /* thin runs on one block: lanes per row, 8, 16 or 32 (0 = 32);
                                fewer lanes let one FP64 instruction serve several rows
                                (default 0) */
} rw_options;

typedef struct rw_context rw_context;
typedef struct rw_factor rw_factor;

/* Read-only view of a factor.  All arrays are device pointers owned by the
 * factor (valid until rw_factor_destroy). */
typedef struct {
    int32_t n;
    int64_t nnz;               /* stored entries of Y (strict lower) */
    const int64_t* y_row_ptr;  /* [n+1] */
    const int32_t* y_col;      /* [nnz], ascending, < row */
    const double* y_val;       /* [nnz] */
    const double* d;           /* [n] */
    const int64_t* yt_row_ptr; /* Y^T in CSR: row i holds (k, Y_ki), k > i, ascending */
    const int32_t* yt_col;
    const double* yt_val;
    const float* y_val32;      /* FP32 copies (NULL unless store_fp32) */
    const float* yt_val32;
    const float* d32;
    const uint32_t* walks;     /* [n] M'_k: walks from row k (0 for exact rows); with reuse the
                                  simulated walks plus the sub-walks that start at k */
    const uint64_t* visits;    /* [n] J'_k: visits to k by walks from k, start included */
    const uint32_t* ground;    /* [n] G'_k: walks from k absorbed at ground */
    const int32_t* walk_rows;  /* [n_walk_rows] rows that ran walks, ascending */
    const int64_t* walk_base;  /* [n_walk_rows+1] first record of each walk row */
    const int32_t* records;    /* [2*total_walks] (end, returns|length) or NULL; end -1 = ground */
    int32_t n_walk_rows;
    int64_t total_walks;       /* simulated walks */
    uint64_t total_hops;       /* sum of walk lengths (hops), first step included */
    int32_t fwd_levels;        /* depth of the DAG of Y z = v */
    int32_t bwd_levels;        /* depth of the DAG of Y^T w = r */
    float phase_ms[8];         /* tables, walk, merge, emit, transpose, levels, fp32, total */
    int64_t kernel_launches;   /* kernels launched by the build */
    int64_t extra_walks;       /* walk reuse: sub-walks counted besides the simulated walks */
    const int32_t* fwd_order;  /* [n] rows of Y z = v by level (level 0 first; any order inside a level) */
    const int64_t* fwd_level_ptr; /* [fwd_levels+1] level l = fwd_order[ptr[l] .. ptr[l+1]) */
    const int32_t* bwd_order;  /* the same for Y^T w = r */
    const int64_t* bwd_level_ptr;
} rw_factor_desc;

typedef struct {
    int32_t iterations;        /* max over right-hand sides */
    double rel_residual;       /* max over right-hand sides of ||b - A x|| / ||b|| (true) */
    float solve_ms;            /* device time of the solve */
    float spmv_ms;             /* device time in A p products (summed over iterations) */
    float bwd_ms;              /* device time in the Y^T w = r solves */
    float fwd_ms;              /* device time in the Y z = w / D solves */
    int64_t kernel_launches;   /* kernels launched by the call */
} rw_pcg_stats;

/* Fill *opt with the defaults listed in rw_options. */
void rw_options_default(rw_options* opt);

/* Create a context on the current device.  stream: cudaStream_t (NULL = the
 * legacy default stream).  alloc/free: both NULL for cudaMallocAsync /
 * cudaFreeAsync on the stream.  opt may be NULL (defaults). */
rw_status rw_context_create(rw_context** out, void* stream, rw_alloc_fn alloc, rw_free_fn free_fn,
                            void* user, const rw_options* opt);
void rw_context_destroy(rw_context* ctx);

/* Precondition step of Algorithm 1 with a uniform budget: walks_per_row walks
 * from every row that has an upper neighbour (rows without one are exact and
 * use no walks, Sec. 5.2).  Draw s of walk w from row k is word (s mod 4) of
 * Philox-4x32-10 with counter (s/4, w, k, tag) and key (lo32(seed), hi32(seed)),
 * tag = (matrix_index << 2), matrix_index = 0 here.  Entries with
 * |Y_ki| < drop_tol are dropped (drop_tol >= 0; 0 keeps every entry).
 * On success *out receives a new factor (rw_factor_destroy releases it). */
rw_status rw_build_factor(rw_context* ctx, const rw_csr* A, uint32_t walks_per_row, uint64_t seed,
                          double drop_tol, rw_factor** out);

/* Same with per-row budgets: d_budget[k] walks from row k (device, [n]; read
 * only for rows with an upper neighbour, each of which needs >= 1). */
rw_status rw_build_factor_budget(rw_context* ctx, const rw_csr* A, const uint32_t* d_budget,
                                 uint64_t seed, double drop_tol, rw_factor** out);

/* Batched precondition step: factors of nmat matrices (As: host array of
 * device CSRs) whose walks all run in ONE persistent kernel launch, with work
 * stealing across rows of all matrices.  Matrix m draws with tag (m << 2) and
 * key seeds[m] (host array), so its factor equals rw_build_factor with matrix
 * index m.  d_budgets: host array of nmat device budget pointers (an entry or
 * the whole array may be NULL: uniform walks_per_row).  outs[m] receive the
 * factors (each released by rw_factor_destroy).  Per-walk records are not
 * kept for batched builds.  On error no factor is returned. */
rw_status rw_build_factor_batched(rw_context* ctx, int32_t nmat, const rw_csr* As,
                                  const uint32_t* const* d_budgets, uint32_t walks_per_row,
                                  const uint64_t* seeds, double drop_tol, rw_factor** outs);

rw_status rw_factor_view(const rw_factor* F, rw_factor_desc* desc);
void rw_factor_destroy(rw_factor* F);

/* Solve step of Algorithm 1: PCG with M = Y^T diag(D) Y for nrhs right-hand
 * sides at once (1 <= nrhs <= 16).  d_b, d_x: node-major [n, nrhs] FP64
 * (entry i of right-hand side r at i*nrhs + r).  x starts at 0.  Each
 * right-hand side stops when its true residual ||b - A x||_2 < tol ||b||_2
 * (the tolerance of the paper's Sec. 6); tol = 0 runs exactly max_iter
 * iterations.  prec = RW_FP32_MIXED: FP32 vectors, SpMV, factor and triangular
 * solves; FP64 dot products, alpha/beta and x, and the residual replaced by an
 * FP64 b - A x every refine_every iterations.  The FP32 SpMV applies A in
 * excess + difference form, e_i x_i + sum_{j != i} A_ij (x_j - x_i) with the
 * FP32 excess e_i = A_ii + sum_j A_ij computed in FP64, so rounding perturbs
 * edge weights and excesses relatively and a weakly grounded matrix keeps its
 * near-null space in FP32.  Returns RW_ERR_NO_CONVERGENCE
 * (x still written) if some right-hand side did not reach tol in max_iter.
 * h_iters/h_relres (host, [nrhs], may be NULL) receive per right-hand side
 * iterations and true relative residuals. */
rw_status pcg_solve(rw_context* ctx, const rw_csr* A, const rw_factor* F, const double* d_b,
                    double* d_x, int32_t nrhs, double tol, int32_t max_iter, rw_precision prec,
                    rw_pcg_stats* stats, int32_t* h_iters, double* h_relres);

/* pcg_solve for nmat matrices (host arrays of matrices, factors, and device
 * right-hand-side / solution pointers), each with nrhs node-major right-hand
 * sides.  stats: host [nmat] (may be NULL); h_iters/h_relres: host
 * [nmat * nrhs] (may be NULL).  Returns RW_ERR_NO_CONVERGENCE if any right-hand
 * side missed tol, the first other error otherwise.  Same as rw_batch_create +
 * pcg_solve_batch + rw_batch_destroy. */
rw_status pcg_solve_batched(rw_context* ctx, int32_t nmat, const rw_csr* As,
                            const rw_factor* const* Fs, const double* const* d_b,
                            double* const* d_x, int32_t nrhs, double tol, int32_t max_iter,
                            rw_precision prec, rw_pcg_stats* stats, int32_t* h_iters,
                            double* h_relres);

/* Batched solves.  A batch joins nmat matrices and their factors into one
 * block-diagonal system: concatenated CSR arrays (rows of matrix m offset by
 * the sizes of matrices 0..m-1), concatenated factors, and one level schedule
 * for each triangular solve over all factors (its depth is the largest single
 * depth).  Each PCG iteration (Algorithm 1) then runs one SpMV, one backward
 * and one forward solve and a few vector kernels for every matrix and
 * right-hand side at once; alpha, beta and the stopping test are per
 * (matrix, right-hand side), computed in FP64 from per-matrix sums in a fixed
 * order, so every system follows the same iterates as pcg_solve on its own
 * matrix up to rounding.  With rw_options.graphs the iteration is captured
 * once in a CUDA graph and replayed; the host reads one flag word per
 * iteration.  A batch of several matrices copies what it needs (it does not
 * reference the matrices or factors afterwards); a batch of one matrix uses
 * that matrix and factor in place, so both must outlive it.  Its arrays are
 * allocated through the context.
 * Limits: sum of n and sum of nnz(A) below 2^31. */
typedef struct rw_batch rw_batch;
rw_status rw_batch_create(rw_context* ctx, int32_t nmat, const rw_csr* As, const rw_factor* const* Fs,
                          rw_batch** out);
void rw_batch_destroy(rw_batch* B);
/* Combined size, stored factor entries and the depths of the two solves. */
rw_status rw_batch_info(const rw_batch* B, int32_t* n_total, int64_t* nnz_y, int32_t* fwd_levels,
                        int32_t* bwd_levels);
/* pcg_solve over the batch: d_b[m], d_x[m] as in pcg_solve_batched.  stats
 * (host [nmat], may be NULL): per matrix the iterations and true residual
 * (max over its right-hand sides), and the device time and kernel launches of
 * the whole call. */
rw_status pcg_solve_batch(rw_context* ctx, rw_batch* B, const double* const* d_b, double* const* d_x,
                          int32_t nrhs, double tol, int32_t max_iter, rw_precision prec,
                          rw_pcg_stats* stats, int32_t* h_iters, double* h_relres);

/* ---- Factor files and orderings -------------------------------------------
 * rw_factor_save writes the factor's rows (Y in CSR, D, and the counters M', J',
 * G' of Sec. 3.1) after a 56-byte header ("RWPCFAC1", version 1, n, walk rows,
 * nnz(Y), walks, hops, levels), followed by the SHA-256 of the payload.
 * rw_factor_load reads such a file, checks the digest and the row structure,
 * and rebuilds the transpose, levels, FP32 copies and solve schedules on the
 * context's device (RW_ERR_ARG for a missing, truncated, foreign or corrupted
 * file).  The loaded factor equals the saved one in every array. */
rw_status rw_factor_save(const rw_factor* F, const char* path);
rw_status rw_factor_load(rw_context* ctx, const char* path, rw_factor** out);
/* SHA-256 (FIPS 180-4) of a host buffer (host code, no device work). */
void rw_sha256(const void* data, size_t len, uint8_t out[32]);
/* A seeded random permutation of 0..n-1 (the random symmetric ordering the
 * paper uses, Sec. 5.4): node i gets the rank of its key, word 0 of
 * Philox-4x32-10 with counter (lo32(i), hi32(i), 0, 2) and key (lo32(seed),
 * hi32(seed)), ties by i.  d_perm (device [n]) receives the new index of each
 * old index. */
rw_status rw_random_permutation(rw_context* ctx, int32_t n, uint64_t seed, int32_t* d_perm);
/* B = P A P^T for a permutation d_perm (old index -> new index): row perm[i] of
 * B holds row i of A with columns perm[j], ascending.  d_row_ptr [n+1], d_col
 * and d_val [nnz] are caller-allocated device arrays.  RW_ERR_ARG if d_perm is
 * not a permutation. */
rw_status rw_permute_csr(rw_context* ctx, const rw_csr* A, const int32_t* d_perm, int32_t* d_row_ptr, int32_t* d_col,
                         double* d_val);

/* Schedule autotuner.  Times a fixed list of launch shapes of the
 * preconditioner application and the SpMV on the given factor (or batch) and
 * nrhs random right-hand sides in precision prec -- the sync-free solve, and
 * the level schedule with entry slices per row group, wide-level blocks per
 * SM and cluster runs off / on for levels of up to 256 rows; SpMV entry
 * slices -- and installs the fastest in the context's options
 * (rw_options.solve_mode, wide_slices, solve_blocks_per_sm, cluster_width,
 * spmv_slices), also copied to *out if not NULL.  cache_path (may be NULL): a
 * JSON-lines file; a line whose key matches the device and the problem's
 * shape (log2 n, stored entries per row, depth, nrhs, precision) is used
 * without timing, otherwise the result is appended.  h_ms (host [2], may be
 * NULL): the best preconditioner and SpMV times in ms (0 when read from the
 * cache).  The factor and the results of later solves are unchanged; only
 * their speed depends on these options. */
rw_status rw_autotune(rw_context* ctx, const rw_csr* A, const rw_factor* F, int32_t nrhs, rw_precision prec,
                      const char* cache_path, rw_options* out, float* h_ms);
rw_status rw_batch_autotune(rw_context* ctx, const rw_batch* B, int32_t nrhs, rw_precision prec,
                            const char* cache_path, rw_options* out, float* h_ms);

/* The two latencies that bound a triangular solve's dependency chain (each
 * level waits for a value stored by another SM): *h_l2_ns, one dependent
 * L2-hit load (a relaxed load chasing a 256 KB cyclic permutation, `iters`
 * steps, one thread); *h_handoff_ns, one SM-to-SM hand-off through L2 (two
 * blocks on distinct SMs pass a counter with relaxed stores and polls, `iters`
 * round trips each, averaged over partner SMs 1, n/4, n/2 and n-1 of block 0).
 * Measurement only: nothing else in the library depends on it.  Synchronous.
 * Errors: RW_ERR_ARG (iters outside [1, 2^20], null outputs), RW_ERR_TIMEOUT (a
 * bounded poll gave up), RW_ERR_ALLOC, RW_ERR_CUDA. */
rw_status rw_probe_latency(rw_context* ctx, int32_t iters, double* h_handoff_ns, double* h_l2_ns);

/* Random-gather throughput of the device memory level that holds a buffer of
 * buffer_bytes (the L2 for a buffer well inside it, HBM for a larger one):
 * threads load aligned units of access_bytes (32, 64 or 128) from uniformly
 * random units of the buffer, four independent loads in flight per thread,
 * about 2^28 units per launch; *h_gbs receives the accessed bytes per second
 * (GB/s) of the second of two launches.  This is the ceiling of a kernel
 * whose reads are random sectors, such as the walk kernel's table reads.
 * Measurement only; the buffer is allocated through the context and freed
 * before the call returns.  Synchronous.  Errors: RW_ERR_ARG (buffer outside
 * [1 MiB, 128 GiB], another access size, null output), RW_ERR_ALLOC,
 * RW_ERR_CUDA. */
rw_status rw_probe_gather(rw_context* ctx, uint64_t buffer_bytes, int32_t access_bytes, double* h_gbs);

/* z = (Y^T diag(D) Y)^-1 r for nrhs node-major right-hand sides (FP64): the
 * preconditioner application inside pcg_solve (backward solve with Y^T,
 * scaling by 1/D, forward solve with Y).
 * Concurrency: every solve on a factor (this call, rw_precond_apply_static,
 * pcg_solve, rw_precond_apply_ldu, bicgstab_solve) uses the factor's own solve
 * workspace (grid-barrier words and thin-run sums), so two of them on the same
 * factor must not overlap on the GPU (different streams or threads); calls on
 * different factors may. */
rw_status rw_precond_apply(rw_context* ctx, const rw_factor* F, const double* d_r, double* d_z,
                           int32_t nrhs);

/* Same result as rw_precond_apply, without allocating.  The paper has no
 * counterpart: this entry point is for callers that cannot allocate device
 * memory at the moment they apply the preconditioner -- an outer iterative
 * solver calling it once per iteration, code running under a fixed memory
 * budget, or a framework whose allocator must not be re-entered from inside a
 * library call.  It calls no cudaMalloc, cudaFree or allocating routine: the
 * scratch vector of the backward solve lives in a file-scope device array of
 * 2^20 doubles (8 MiB) that every GPU loading the library holds until the
 * process exits.  n * nrhs must not exceed 2^20 (RW_ERR_CAPACITY otherwise).
 * The first call on a device looks up that array's device address (with the
 * device current); make that first call before any stream capture.  Every
 * call synchronises the context stream before it returns (it reads back the
 * device status).  All calls share the one array, which keeps the previous
 * call's contents (this call re-initialises what it reads), so calls that
 * overlap on the GPU -- on different streams or from different threads -- race
 * and must not be issued; the factor's solve workspace is shared as for
 * rw_precond_apply.  The current device must be the context's device. */
rw_status rw_precond_apply_static(rw_context* ctx, const rw_factor* F, const double* d_r,
                                  double* d_z, int32_t nrhs);

/* y = A x for nrhs node-major vectors (FP64). */
rw_status rw_spmv(rw_context* ctx, const rw_csr* A, const double* d_x, double* d_y, int32_t nrhs);

/* ---- Learned walk budget ------------------------------------------------
 * Sec. 5.1 chooses M_k per row so that the mean walk length Xi'_k of the M_k
 * walks from row k is within a relative margin Delta of its expectation at
 * confidence alpha (Eq. lengthdelta), i.e. M*_k = (z_alpha sigma_k /
 * (Delta Xi'_k))^2, with a lower bound on M_k.  Here a small network predicts
 * log((sigma_k / Xi'_k)^2) from per-row graph features (trained on pilot-walk
 * statistics), and the normaliser turns the predicted relative needs into
 * integer budgets with a requested mean and minimum, i.e. it fixes
 * (z_alpha / Delta)^2 from the walk count one is willing to spend.          */

#define RW_NUM_FEATURES 12
#define RW_FEATURE_STRIDE 16   /* floats per feature row; entries 12..15 are 0 */
#define RW_MLP_PARAMS 5313     /* 64*16 + 64 + 64*64 + 64 + 64 + 1 */

typedef struct rw_mlp rw_mlp;

/* Per-row graph features into d_feat [n][RW_FEATURE_STRIDE] (FP32, computed
 * in FP64): 0 log(1+degree), 1 upper/degree, 2 lower/degree, 3 excess/A_kk,
 * 4 -S_k/A_kk (S_k: sum of the row's upper entries), 5 entropy of the
 * transition probabilities -A_kj/(sum of the row's off-diagonal weights),
 * 6 largest weight / weight sum, 7 k/(n-1), 8 mean over neighbours c of
 * (row sum of c)/A_cc, 9 log(1 + mean neighbour degree), 10 log(1 + sum over
 * upper neighbours c of the entries of row c with column > k), 11 log A_kk.
 * A must be an R-matrix in rw_csr form (not re-validated here). */
rw_status rw_row_features(rw_context* ctx, const rw_csr* A, float* d_feat);

/* Pilot walks: pilot_walks (>= 2) walks from every walk row under the walk
 * kind 1 (Philox counter word 3 = 1; rw_build_factor uses kind 0), and per row
 * the mean and sample standard deviation of a per-walk quantity, the label
 * log((sd/mean)^2 + 1e-6) and has_k = 1 (rows without walks: all four 0).
 * quantity 0: the walk length in hops (Xi'_k of Sec. 5.1); quantity 1: the
 * visits to the start row, 1 + returns (J'_k / M'_k of Sec. 3.1, the
 * "expected number of returns" that Sec. 5.1 names as an alternative
 * b-independent quantity; it sets D_kk in Eq. newz).  quantity 2: the
 * visits' statistics with the cost-aware label
 * (log((sd/mean)^2 + 1e-6) - log Xi'_k) / 2 from the same walks recorded twice:
 * exp(label) is then the allocation of a fixed hop count (walks cost Xi'_k
 * hops each) that minimises the sum of the rows' relative variances
 * (M_k proportional to sd_k / (mean_k sqrt(Xi'_k))).  Outputs are device
 * arrays [n].  Errors as for rw_build_factor (RW_ERR_NOT_RMATRIX,
 * RW_ERR_WALK_CAP, ...). */
rw_status rw_pilot_stats(rw_context* ctx, const rw_csr* A, uint32_t pilot_walks, uint64_t seed, int32_t quantity,
                         float* d_mean, float* d_sd, float* d_label, float* d_has);

/* The network 12 -> 64 -> 64 -> 1 (ReLU): x = bf16((f - mu) * inv_sd),
 * h1 = bf16(relu(W1 x + b1)), h2 = relu(W2 h1 + b2), y = w3.h2 + b3; W1 and W2
 * are used in BF16 with FP32 accumulation (tensor cores), the master copy is
 * FP32.  Parameter vector layout (RW_MLP_PARAMS floats): W1 [64][16]
 * (output-major; columns 12..15 ignored), b1 [64], W2 [64][64] (output-major),
 * b2 [64], w3 [64], b3.  Standardisation vector (32 floats): mu [16],
 * inv_sd [16].  rw_mlp_create draws He-uniform weights from seed (zero biases,
 * mu = 0, inv_sd = 1).  The model lives on the context's device; destroy it
 * before the context. */
rw_status rw_mlp_create(rw_context* ctx, uint64_t seed, rw_mlp** out);
void rw_mlp_destroy(rw_mlp* M);
/* Host copies: h_params/h_norm receive the current values (if not NULL),
 * after h_set_params/h_set_norm (if not NULL) were installed; setting the
 * parameters resets the Adam state. */
rw_status rw_mlp_params(rw_mlp* M, float* h_params, float* h_norm, const float* h_set_params,
                        const float* h_set_norm);
/* d_out[r] = y of feature row r, r < nrows (d_feat as rw_row_features). */
rw_status rw_mlp_predict(rw_context* ctx, const rw_mlp* M, const float* d_feat, int64_t nrows,
                         float* d_out);
/* Gradient (h_grad [RW_MLP_PARAMS], host) of the loss (1/B) sum_r (y_r -
 * label_r)^2 over the B = nrows feature rows listed in d_rows (device uint32
 * indices into d_feat/d_label), and the loss (h_loss, optional).  The backward
 * pass rounds dL/dh2 to BF16 for the product with W2 (tensor cores); weight
 * gradients accumulate in FP32 in a fixed order (deterministic). */
rw_status rw_mlp_gradient(rw_context* ctx, rw_mlp* M, const float* d_feat, const float* d_label,
                          const uint32_t* d_rows, int64_t nrows, float* h_grad, float* h_loss);
/* Adam training (beta 0.9/0.999, eps 1e-8, learning rate lr) on the rows with
 * d_mask[r] > 0, for `epochs` passes of floor(rows/batch) mini-batches in a
 * seeded shuffled order.  set_norm != 0 first sets mu/inv_sd to the masked
 * rows' feature means and inverse standard deviations.  h_epoch_loss
 * (optional, [epochs]) receives each epoch's mean squared error. */
rw_status rw_mlp_train(rw_context* ctx, rw_mlp* M, const float* d_feat, const float* d_label,
                       const float* d_mask, int64_t nrows, int32_t epochs, int32_t batch, float lr,
                       uint64_t seed, int32_t set_norm, float* h_epoch_loss);

/* Integer walk budgets from relative needs w_k >= 0 (device [n]): over the
 * walk rows (rows with an upper neighbour; the others get 0), with
 * T = floor(mean_budget * walk_rows + 1/2):
 *   quota q_k(s) = min(min(T, 2^31), max(min_budget, s w_k)),
 *   V_k = round-half-even(q_k 2^20) (fixed point), s found by a fixed doubling
 *   and bisection search for the largest sum_k V_k(s) not above T 2^20;
 *   budget_k = floor(V_k 2^-20) + R / walk_rows + [rank_k < R mod walk_rows],
 *   R = T - sum floor, ranks by fractional part descending then k ascending
 *   (largest-remainder apportionment).
 * The budgets sum to T exactly and each is at least min_budget.  Every step is
 * exact arithmetic, so the result is reproducible bit for bit.  Errors:
 * RW_ERR_ARG for min_budget < 1, mean_budget < min_budget or > 2^31, T > 2^40,
 * or a negative, infinite or NaN weight on a walk row. */
rw_status rw_budget_normalize(rw_context* ctx, const rw_csr* A, const float* d_weight,
                              double mean_budget, uint32_t min_budget, uint32_t* d_budget);
/* Features -> network -> w_k = exp(y_k) (FP32, y clamped to [-60, 60]) ->
 * rw_budget_normalize.  d_budget [n] feeds rw_build_factor_budget. */
rw_status rw_budget_predict(rw_context* ctx, const rw_csr* A, const rw_mlp* M, double mean_budget,
                            uint32_t min_budget, uint32_t* d_budget);

/* Adaptive walk counts of Sec. 5.1 (Eq. lengthdelta).  The paper keeps
 * adding walks from row k until Delta Xi' sqrt(M_k) / sigma > z, where Xi' and
 * sigma are the mean and sample standard deviation of the row's walk lengths
 * and z = Q^-1((1 - alpha)/2) for confidence alpha.  Each walk row is first
 * decided after min_walks factor walks; a row failing Delta^2 Xi'^2 M > z^2
 * sigma^2 (with M < max_walks) grows to max(M + 1, ceil(z^2 sigma^2 /
 * (Delta^2 Xi'^2))), capped at max_walks, and is decided again with that many
 * walks; at most max_rounds decisions per row.  The GPU runs the rows in launch
 * rounds that run rw_options.adapt_ahead percent of a row's next decision
 * point past it, so one round can hold several decisions of a row; walks past
 * the final count are discarded.  Walks are the factor walks (walk kind 0) of matrix index 0 with
 * `seed`, so rw_build_factor_budget(seed, d_budget) afterwards consists of
 * exactly the walks that fixed the counts.  Length sums are exact 64-bit
 * integers and the test is FP64 with each operation rounded once, so the
 * counts are deterministic.
 *   d_budget [n] device uint32, written: M_k for walk rows, 0 for the others.
 *   h_rounds host, optional: the most decisions any row took (the rounds of
 *   a schedule that decides every row once per round).
 * Errors: RW_ERR_ARG (delta, z <= 0; min_walks < 2; max_walks < min_walks or
 * > 65535; max_rounds < 1), RW_ERR_NOT_RMATRIX, RW_ERR_WALK_CAP (a walk hit
 * rw_options.max_steps), RW_ERR_ALLOC, RW_ERR_CUDA.  Synchronous. */
rw_status rw_adaptive_budget(rw_context* ctx, const rw_csr* A, uint64_t seed, double delta, double z,
                             uint32_t min_walks, uint32_t max_walks, int32_t max_rounds, uint32_t* d_budget,
                             int32_t* h_rounds);

/* Nonsymmetric matrices (Sec. 7.1).  The walk game needs only diagonal
 * dominance by rows, so the game on A and the game on A^T (A dominant by rows
 * and by columns, negative off-diagonals) give two factors: with F_A built on
 * A and F_AT on A^T, A ~= Y_AT^T diag(D) Y_A (Y_A ~ the rev-LDU's U part of
 * the paper's Eq. y2, Y_AT^T its L part by Eq. y3, D from the game on A).
 * rw_csr_transpose writes B = A^T (device arrays of the caller: row_ptr [n+1],
 * col and val [nnz]; columns ascending in each row); synchronous.
 * rw_precond_apply_ldu applies z = (Y_AT^T D Y_A)^-1 r (backward solve with
 * Y_AT^T, scaling by 1/D, forward solve with Y_A), nrhs <= 16, node-major, with
 * the context's solve schedule options.
 * bicgstab_solve solves A x = b (one right-hand side, FP64) by BiCGSTAB with
 * that preconditioner on the right, from x = 0, until the true residual
 * ||b - A x|| < tol ||b||; stats: iterations, true relative residual, time.
 * Errors: RW_ERR_ARG (sizes or factors that do not match), RW_ERR_NO_CONVERGENCE
 * (max_iter reached; x holds the last iterate), RW_ERR_BREAKDOWN (a BiCGSTAB
 * scalar became zero), RW_ERR_ALLOC, RW_ERR_CUDA. */
rw_status rw_csr_transpose(rw_context* ctx, const rw_csr* A, int32_t* d_row_ptr, int32_t* d_col, double* d_val);
rw_status rw_precond_apply_ldu(rw_context* ctx, const rw_factor* F_A, const rw_factor* F_AT, const double* d_r,
                               double* d_z, int32_t nrhs);
rw_status bicgstab_solve(rw_context* ctx, const rw_csr* A, const rw_factor* F_A, const rw_factor* F_AT,
                         const double* d_b, double* d_x, double tol, int32_t max_iter, rw_pcg_stats* stats);

const char* rw_status_string(rw_status s);
const char* rw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RWPC_H */
