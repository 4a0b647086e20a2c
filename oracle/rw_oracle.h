/*
 * rw_oracle.h -- CPU oracle for the random-walk incomplete LDL^T preconditioner.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  This is a plain, slow restatement of
 * the method of Qian & Sapatnekar, "Stochastic Preconditioning for Iterative
 * Linear Equation Solvers", used only by the tests, by the smoke check and by
 * the CPU-baseline leg of the benchmark.  Everything is single-threaded except
 * orc_factor_build_mt, which runs the rows of the plain build on several host
 * threads (for timing on all cores and for full-size parity inputs).  It shares
 * no code with the CUDA library and must never be linked into it.
 *
 * Index convention: 0-based.  Walks started at row k treat rows 0..k-1 as homes
 * (Sec. 2.2.1) plus the virtual ground reached through the diagonal excess
 * (Sec. 2.1, Eq. map).  The exported factor satisfies A ~= Y^T diag(D) Y with Y
 * unit lower triangular (strict lower part stored), which is the paper's
 * L_rev(A) = rev(Y)^T and D_rev(A) = rev(D) (Eqs. y and d) in the original index
 * order.
 *
 * Return codes: 0 ok, -1 bad argument, -2 not an R-matrix, -3 a walk reached the
 * step cap, -4 out of memory, -5 PCG did not converge, -6 PCG breakdown.
 */
#ifndef RW_ORACLE_H
#define RW_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Draw number s of walk w from row k: word (s mod 4) of
 * Philox(ctr = {s/4, w, k, (matrix_index << 2) | tag}, key = {lo32(seed), hi32(seed)}). */
uint32_t orc_draw(uint64_t seed, uint32_t matrix_index, uint32_t tag, uint32_t k,
                  uint32_t w, uint64_t s);

/* Integer transition thresholds of row l (Sec. 2.1, Eq. map): t_m for the m-th
 * off-diagonal entry in ascending column order.  Returns the number written. */
int32_t orc_row_thresholds(const int32_t* rowptr, const int32_t* col, const double* val,
                           int32_t l, uint32_t* t_out);

/* Validate A as an R-matrix in the form the method needs. 0 or -2. */
int orc_validate(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val);

typedef struct orc_factor orc_factor;

/*
 * Build the factor from walks (Algorithm 1, "Precondition").
 *   budget[k]   walks from row k (read only for rows with an upper neighbour)
 *   mode        0: one-step-exact walks (Sec. 5.2, Eqs. newy/newz)
 *               1: the same plus walk reuse (Sec. 5.3, Algorithm 2)
 *   rows/nrows  optional ascending subset of rows to compute (mode 0 only; rows
 *               are independent, Sec. 4); the other rows are left empty with D = 0.
 *   rec_end/rec_ret/rec_len  optional per-walk records (end node, -1 = ground;
 *               returns to the start row; hops), in walk order (rows ascending,
 *               walk index ascending); capacity rec_cap.
 */
int orc_factor_build(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const uint32_t* budget, uint64_t seed, uint32_t matrix_index, uint32_t tag,
                     double drop_tol, uint64_t max_steps, int32_t mode,
                     const int32_t* rows, int32_t nrows,
                     int32_t* rec_end, uint32_t* rec_ret, uint32_t* rec_len, int64_t rec_cap,
                     orc_factor** out);
/* orc_factor_build (mode 0, no records) on nthreads host threads: rows are
 * independent (Sec. 4), so chunks of rows run concurrently and are joined in
 * row order; the factor equals the single-thread build bit for bit. */
int orc_factor_build_mt(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                        const uint32_t* budget, uint64_t seed, uint32_t matrix_index, uint32_t tag,
                        double drop_tol, uint64_t max_steps, const int32_t* rows, int32_t nrows,
                        int32_t nthreads, orc_factor** out);
int64_t orc_factor_nnz(const orc_factor* f);
void orc_factor_get(const orc_factor* f, int64_t* rowptr, int32_t* col, double* val, double* D,
                    uint64_t* M, uint64_t* J, uint64_t* G, uint64_t* hops);
void orc_factor_free(orc_factor* f);

/* Algorithm 2 on one explicit walk sequence k_1..k_G (1-based node labels as in
 * the paper's example).  Adds the extracted sub-walks to dM[n+1], dJ[n+1] and
 * writes the (start, end) pairs of the extracted walks to hs/he (capacity cap).
 * Returns the number of extracted walks (the root walk itself is not included). */
int32_t orc_reuse_trace(const int32_t* seq, int32_t len, int32_t nlabels,
                        int64_t* dM, int64_t* dJ, int32_t* hs, int32_t* he, int32_t cap);

/* z = (Y^T diag(D) Y)^-1 r in FP64: backward substitution with Y^T, scaling by
 * 1/D, forward substitution with Y (the preconditioner of Algorithm 1). */
int orc_precond_apply(int32_t n, const int64_t* Yrp, const int32_t* Ycol, const double* Yval,
                      const double* D, const double* r, double* z);

/*
 * Preconditioned conjugate gradients with M = Y^T D Y (Algorithm 1, "solve").
 * One right-hand side.  mixed=0: FP64 throughout.  mixed=1: FP32 vectors, SpMV,
 * factor and triangular solves; FP64 dot products, alpha/beta and x; the residual
 * is recomputed in FP64 every refine_every iterations.  The FP32 SpMV applies A
 * in excess + difference form (FP32 off-diagonals A_ij and FP32 excesses
 * e_i = A_ii + sum_j A_ij: y_i = e_i x_i + sum_j A_ij (x_j - x_i)).  Stops when the true
 * residual ||b - A x|| < tol ||b||; tol = 0 runs exactly max_iter iterations.
 */
int orc_pcg(int32_t n, const int32_t* Arp, const int32_t* Acol, const double* Aval,
            const int64_t* Yrp, const int32_t* Ycol, const double* Yval, const double* D,
            const double* b, double* x, double tol, int32_t max_iter, int32_t mixed,
            int32_t refine_every, int32_t* iters_out, double* relres_out);

/* Adaptive walk counts of Sec. 5.1 (Eq. lengthdelta), in rounds; see rw_oracle.c. */
int orc_adaptive_budget(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                        uint64_t seed, uint32_t matrix_index, double delta, double z,
                        uint32_t min_walks, uint32_t max_walks, int32_t max_rounds,
                        uint64_t max_steps, uint32_t* budget, int32_t* rounds_out);

#ifdef __cplusplus
}
#endif
#endif
