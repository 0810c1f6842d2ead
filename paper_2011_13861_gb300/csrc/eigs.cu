// Eigensolver driver: thick-restart block Lanczos with full float64 re-orthogonalisation.
//
// The paper solves the standard-form problem A~' v' = lambda v' with implicitly restarted
// Lanczos (Sec. 4.4.2).  Here the same Krylov iteration is organised as a thick restart
// (equivalent to implicit restarting with exact shifts) in blocks of b vectors, so that one
// on-the-fly kernel evaluation serves b right-hand sides:
//
//   expansion:  W = A~' Q_j;  H = V^T W;  W -= V H (twice, classical Gram-Schmidt);
//               W = Q_{j+1} R (block Cholesky-QR, twice);  T holds V^T A~' V
//   restart:    T = S Theta S^T (Jacobi);  keep p Ritz vectors Y = V S_{:,1:p};
//               A~' Y = Y Theta_p + F S_{m-b:m,1:p}  with F the last orthogonalised W,
//               so the new basis is [Y, orth(F)] with T = [Theta_p, (R S_last)^T; R S_last, .]
//   residual:   ||A~' y_i - theta_i y_i|| = ||F s_i^{last}||  (Lanczos estimate), checked at the
//               end with an explicit float64 application when requested.
//
// Method 1 ("mixed") runs the iteration with the float32 stage-5 kernel until the estimates
// reach tol_low, then continues from the float32 Ritz vectors in one wide block (b = number
// of kept vectors), which converges in a few block steps: the first block takes the float64
// (-class) operator, the correction blocks after it the float32 one (see run_phase).  The
// float32 phase orthogonalises with one pass of Gram-Schmidt and of Cholesky-QR and forms its
// basis products in double-float on the float32 pipe; the polish keeps two float64 passes.
// Everything stays on the device; per restart the host reads back the Ritz values and
// residual estimates of the wanted pairs (a few hundred bytes).
#include <math.h>

#include <cmath>

#include <algorithm>
#include <chrono>
#include <vector>

#include "kl_internal.h"

namespace kl {
namespace {

// the float32-class operators' relative error on the smooth vectors that correction blocks
// contribute to Ritz vectors (their rounding errors average over the ~1e3-1e5 terms of a row:
// 3e-7 to 6e-7 of the largest entry for random vectors, far less for smooth ones)
constexpr double kEps32 = 1e-7;

struct Eig {
    kl_handle h;
    cudaStream_t s;
    int64_t N;
    int mmax;    // capacity of the basis
    int bmax;    // capacity of a block
    kl::DevBuf bV, bW, bY, bT, bTc, bS, bSw, bTheta, bH, bH2, bG, bR, bR1, bRinv, bRtmp, bPart, bEst, bFlag, bSweeps;
    kl::DevBuf bAV, bY2;   // A~'V (the operator products of the basis, kept through restarts)
    double* AV() { return static_cast<double*>(bAV.ptr); }
    double* Y2() { return static_cast<double*>(bY2.ptr); }
    double* V() { return static_cast<double*>(bV.ptr); }
    double* W() { return static_cast<double*>(bW.ptr); }
    double* Y() { return static_cast<double*>(bY.ptr); }
    double* T() { return static_cast<double*>(bT.ptr); }
    double* S() { return static_cast<double*>(bS.ptr); }
    double* Sw() { return static_cast<double*>(bSw.ptr); }
    double* Theta() { return static_cast<double*>(bTheta.ptr); }
    double* H() { return static_cast<double*>(bH.ptr); }
    double* H2() { return static_cast<double*>(bH2.ptr); }
    double* G() { return static_cast<double*>(bG.ptr); }
    double* R() { return static_cast<double*>(bR.ptr); }
    double* R1() { return static_cast<double*>(bR1.ptr); }
    double* Rinv() { return static_cast<double*>(bRinv.ptr); }
    double* Rtmp() { return static_cast<double*>(bRtmp.ptr); }
    double* Part() { return static_cast<double*>(bPart.ptr); }
    double* Est() { return static_cast<double*>(bEst.ptr); }
    int* Flag() { return static_cast<int*>(bFlag.ptr); }
    int* Sweeps() { return static_cast<int*>(bSweeps.ptr); }
    int maxparts = 0;
    // statistics
    int applies = 0, applies64 = 0, appliesdf = 0, appliestc64 = 0, appliestc32 = 0, block_applies = 0;
    uint64_t rng_offset = 0;
    uint64_t seed = 1;

    ~Eig() {
        kl::DevBuf* all[] = {&bV, &bW, &bY, &bT, &bTc, &bS, &bSw, &bTheta, &bH, &bH2, &bG, &bR, &bR1,
                             &bRinv, &bRtmp, &bPart, &bEst, &bFlag, &bSweeps, &bAV, &bY2};
        for (auto* b : all) release(*b);
    }

    kl_status alloc(int m, int b) {
        mmax = m;
        bmax = b;
        const size_t N8 = size_t(N) * sizeof(double);
        KL_TRY(ensure(bV, N8 * (m + b)));
        KL_TRY(ensure(bW, N8 * std::max(b, 64)));
        KL_TRY(ensure(bY, N8 * std::max(m, 64)));
        KL_TRY(ensure(bAV, N8 * (m + b)));
        KL_TRY(ensure(bY2, N8 * std::max(m, 64)));
        KL_TRY(ensure(bT, sizeof(double) * m * m));
        KL_TRY(ensure(bTc, sizeof(double) * m * m));
        KL_TRY(ensure(bS, sizeof(double) * m * m));
        KL_TRY(ensure(bSw, 4 * sizeof(double) * m * m));
        KL_TRY(ensure(bTheta, sizeof(double) * m));
        KL_TRY(ensure(bH, sizeof(double) * m * b));
        KL_TRY(ensure(bH2, sizeof(double) * m * b));
        KL_TRY(ensure(bG, sizeof(double) * b * b));
        KL_TRY(ensure(bR, sizeof(double) * b * b));
        KL_TRY(ensure(bR1, sizeof(double) * b * b));
        KL_TRY(ensure(bRinv, sizeof(double) * b * b));
        KL_TRY(ensure(bRtmp, sizeof(double) * b * b));
        maxparts = gram_parts(N);
        KL_TRY(ensure(bPart, sizeof(double) * size_t(maxparts) * std::max(192 * 32, 64 * 64)));
        KL_TRY(ensure(bEst, sizeof(double) * (m + 64)));
        KL_TRY(ensure(bFlag, sizeof(int) * 4));
        KL_TRY(ensure(bSweeps, sizeof(int) * 4));
        return KL_OK;
    }

    kl_status apply(int prec, const double* Q, double* Wout, int b) {
        KL_TRY(apply_impl(h, prec, Q, N, Wout, N, b, s));
        applies += b;
        if (prec == KL_P_FP64) applies64 += b;
        if (prec == KL_P_DF64) appliesdf += b;
        if (prec == KL_P_TC64) appliestc64 += b;
        if (prec == KL_P_TC32) appliestc32 += b;
        block_applies += 1;
        return KL_OK;
    }

    // One pass of classical Gram-Schmidt and of Cholesky-QR instead of two (a phase whose own
    // operator is float32-accurate: the orthogonality a single pass leaves, about eps64 times
    // the norm drop ||W|| / ||W - V H|| or times cond(W)^2, is far below what it resolves)
    bool one_pass = false;
    // the products of the basis: float64, or double-float on the float32 pipe where one_pass (the
    // float32 phase, whose operator resolves neither)
    cudaError_t gram(const double* A, int64_t lda, int p, const double* B, int64_t ldb, int q, double* out, int ldo) {
        return one_pass ? launch_gram_df(A, lda, p, B, ldb, q, N, out, ldo, Part(), maxparts, s)
                        : launch_gram(A, lda, p, B, ldb, q, N, out, ldo, Part(), maxparts, s);
    }
    cudaError_t gemm(double alpha, const double* A, int64_t lda, int p, const double* B, int ldb, int q, double beta,
                     double* C, int64_t ldc) {
        return one_pass ? launch_gemm_tall_df(alpha, A, lda, N, p, B, ldb, q, beta, C, ldc, s)
                        : launch_gemm_tall(alpha, A, lda, N, p, B, ldb, q, beta, C, ldc, s);
    }
    // where the last run_phase stopped: its basis size and the leading columns whose products
    // were accurate (correction blocks); contam: estimated float32 error (absolute) that earlier
    // cycles' correction blocks left in the kept Ritz vectors' carried products
    int exit_j = 0, exit_acc = 0;
    bool exit_restarted = false;
    double contam = 0.0;

    // max over the first `cols` Ritz vectors of kEps32 ||(A~'V)[:, acc:j] S[acc:j, i]||
    kl_status correction_error(int acc, int j, int cols, std::vector<double>* per_col) {
        const int nlo = j - acc;
        per_col->assign(cols, 0.0);
        if (nlo <= 0 || cols <= 0) return KL_OK;
        cudaError_t e = launch_gemm_tall(1.0, AV() + size_t(acc) * N, N, N, nlo, S() + acc, mmax, cols, 0.0, Y2(), N, s);
        if (e == cudaSuccess) e = launch_gram(Y2(), N, cols, Y2(), N, cols, N, G(), cols, Part(), maxparts, s);
        if (e != cudaSuccess) return cuda_fail(e, "correction products");
        std::vector<double> g(size_t(cols) * cols);
        KL_TRY(host_wait(h, s));
        KL_CUDA(cudaMemcpyAsync(g.data(), G(), g.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        KL_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < cols; ++i) (*per_col)[i] = kEps32 * std::sqrt(std::max(g[size_t(i) * cols + i], 0.0));
        return KL_OK;
    }

    // H (j x b, ld mmax) = V[:, 0:j]^T W ; W -= V H   (twice); returns accumulated H in H()
    kl_status orthogonalize(double* Wb, int b, int j) {
        if (j == 0) return KL_OK;
        cudaError_t e = gram(V(), N, j, Wb, N, b, H(), mmax);
        if (e != cudaSuccess) return cuda_fail(e, "gram");
        e = gemm(-1.0, V(), N, j, H(), mmax, b, 1.0, Wb, N);
        if (e != cudaSuccess) return cuda_fail(e, "update");
        if (one_pass) return KL_OK;
        e = launch_gram(V(), N, j, Wb, N, b, N, H2(), mmax, Part(), maxparts, s);
        if (e != cudaSuccess) return cuda_fail(e, "gram");
        e = launch_gemm_tall(-1.0, V(), N, N, j, H2(), mmax, b, 1.0, Wb, N, s);
        if (e != cudaSuccess) return cuda_fail(e, "update");
        // H += H2 (both stored with ld mmax, j rows, b columns)
        // one launch over the b columns (rows j..mmax-1 of each column are unused scratch)
        e = launch_add_inplace(H(), H2(), int(size_t(mmax) * (b - 1) + j), s);
        if (e != cudaSuccess) return cuda_fail(e, "accumulate");
        return KL_OK;
    }

    // W = Q R with Q orthonormal (CholQR2).  R (b x b, ld b) in R(); Q written to dst (ld N).
    // Returns true in *deficient when the block is numerically rank deficient.
    kl_status cholqr(double* Wb, int b, double* dst, bool* deficient) {
        int flags[2] = {0, 0};
        double* cur = Wb;
        if (one_pass && dst != Wb) {
            cudaError_t e = gram(Wb, N, b, Wb, N, b, G(), b);
            if (e == cudaSuccess) e = launch_chol_inv(G(), b, b, Rinv(), R(), Flag(), s);
            if (e != cudaSuccess) return cuda_fail(e, "chol");
            e = gemm(1.0, Wb, N, b, Rinv(), b, b, 0.0, dst, N);
            if (e != cudaSuccess) return cuda_fail(e, "scale");
            KL_TRY(host_wait(h, s));
            KL_CUDA(cudaMemcpyAsync(flags, Flag(), sizeof(int), cudaMemcpyDeviceToHost, s));
            KL_CUDA(cudaStreamSynchronize(s));
            *deficient = (flags[0] != 0);
            return KL_OK;
        }
        for (int pass = 0; pass < 2; ++pass) {
            cudaError_t e = launch_gram(cur, N, b, cur, N, b, N, G(), b, Part(), maxparts, s);
            if (e != cudaSuccess) return cuda_fail(e, "gram");
            double* Rp = pass == 0 ? R1() : Rtmp();
            e = launch_chol_inv(G(), b, b, Rinv(), Rp, Flag() + pass, s);
            if (e != cudaSuccess) return cuda_fail(e, "chol");
            double* out = (pass == 0) ? Y() : dst;
            e = launch_gemm_tall(1.0, cur, N, N, b, Rinv(), b, b, 0.0, out, N, s);
            if (e != cudaSuccess) return cuda_fail(e, "scale");
            cur = out;
        }
        // R = R2 R1 (upper triangular product), computed as a tiny "tall" product with N = b rows
        // R^T = R1^T R2^T ; use gemm on the transposes: R[i][j] = sum_c R2[i][c] R1[c][j]
        // gemm_tall computes C[r, :] = A[r, :] B with A = R2 (b x b, ld b), B = R1.
        cudaError_t e = launch_gemm_tall(1.0, Rtmp(), b, b, b, R1(), b, b, 0.0, R(), b, s);
        if (e != cudaSuccess) return cuda_fail(e, "R product");
        KL_TRY(host_wait(h, s));
        KL_CUDA(cudaMemcpyAsync(flags, Flag(), 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        KL_CUDA(cudaStreamSynchronize(s));
        *deficient = (flags[0] != 0);
        return KL_OK;
    }

    // CholQR2 of W with the same right factors applied to a companion block C (the operator
    // products of W): dst = W R^{-1}, cdst = C R^{-1}.  dst may equal W and cdst may equal C.
    kl_status cholqr_pair(double* Wb, double* Cb, int b, double* dst, double* cdst, bool* deficient) {
        int flags[2] = {0, 0};
        double* cur = Wb;
        double* ccur = Cb;
        for (int pass = 0; pass < 2; ++pass) {
            cudaError_t e = launch_gram(cur, N, b, cur, N, b, N, G(), b, Part(), maxparts, s);
            if (e != cudaSuccess) return cuda_fail(e, "gram");
            e = launch_chol_inv(G(), b, b, Rinv(), pass == 0 ? R1() : Rtmp(), Flag() + pass, s);
            if (e != cudaSuccess) return cuda_fail(e, "chol");
            double* out = (pass == 0) ? Y() : dst;
            double* cout = (pass == 0) ? Y2() : cdst;
            e = launch_gemm_tall(1.0, cur, N, N, b, Rinv(), b, b, 0.0, out, N, s);
            if (e == cudaSuccess) e = launch_gemm_tall(1.0, ccur, N, N, b, Rinv(), b, b, 0.0, cout, N, s);
            if (e != cudaSuccess) return cuda_fail(e, "scale");
            cur = out;
            ccur = cout;
        }
        KL_TRY(host_wait(h, s));
        KL_CUDA(cudaMemcpyAsync(flags, Flag(), 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        KL_CUDA(cudaStreamSynchronize(s));
        *deficient = (flags[0] != 0 || flags[1] != 0);
        return KL_OK;
    }

    // fresh random directions orthogonal to V[:, 0:j] written into dst (N x b)
    kl_status random_orthonormal(double* dst, int b, int j) {
        for (int attempt = 0; attempt < 3; ++attempt) {
            cudaError_t e = launch_random_block(W(), N, N, b, seed ^ 0xA5A5A5A5ull, rng_offset, s);
            rng_offset += uint64_t(N) * b;
            if (e != cudaSuccess) return cuda_fail(e, "random block");
            KL_TRY(orthogonalize(W(), b, j));
            bool def = false;
            KL_TRY(cholqr(W(), b, dst, &def));
            if (!def) return KL_OK;
        }
        return fail(KL_ERR_NUMERIC, "could not extend the Krylov basis");
    }

    // AV[:, 0:keep] = AV[:, 0:j] S[:, 0:keep]: the products of the new basis (Ritz vectors)
    kl_status rotate_products(int j, int keep) {
        cudaError_t e = launch_gemm_tall(1.0, AV(), N, N, j, S(), mmax, keep, 0.0, Y2(), N, s);
        if (e != cudaSuccess) return cuda_fail(e, "rotate products");
        e = launch_copy_block(Y2(), N, AV(), N, N, keep, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy products");
        return KL_OK;
    }

    kl_status sym_eig(int m) {
        cudaError_t e = launch_sym_eig_ws(T(), mmax, m, Theta(), S(), mmax, Sw(), Sweeps(), s);
        if (e != cudaSuccess) return cuda_fail(e, "small eigensolver");
        return KL_OK;
    }
};

struct Phase {
    int prec;
    int b;
    int m;
    int keep;
    double tol;
    bool early_rr;     // Rayleigh-Ritz after every block step (used for the float64 polish)
    int maxrestart;
    int exit_vecs;     // Ritz vectors left in V[:, 0:exit_vecs] on exit (>= k)
    int prec_next;     // arithmetic of every application after the phase's first (see run_phase)
    bool carry = true; // keep A~'V with the basis (false: a later phase recomputes the products)
    bool skip_first_rr = false;   // no early Rayleigh-Ritz check after the phase's first block
    bool one_pass = false;        // single-pass Gram-Schmidt and Cholesky-QR (Eig::one_pass)
};

// Runs one thick-restart block Lanczos phase.  On entry V[:, 0:j0] holds an orthonormal basis
// whose last b columns form the active block and T[0:j0, 0:j0] = V^T A V is valid for all
// but the active block's column (the next expansion recomputes it).  On exit V[:, 0:k] holds
// the k wanted Ritz vectors, Theta their values and est[] the residual estimates.
//
// Correction blocks in lower precision (P.prec_next != P.prec, the polish of the mixed method):
// only the phase's first application (the float32 phase's Ritz block X) takes P.prec; every
// later block Q_i takes P.prec_next.  The Ritz vectors of span[X, Q_1, ..] are
// y = X s_0 + sum_i Q_i s_i with |s_i| of the order of X's residual, so an operator error eps
// in A Q_i moves their residuals, and the products carried with them, by about
// eps ||A|| |s_i|: 1e-7 x 1e-6 of ||A|| for a float32 operator after a float32 phase that
// stopped at 1e-6, far below a 1e-8 tolerance.  What must stay in the accurate precision is
// the coupling of the accurate columns (X, or the Ritz vectors kept at a restart, whose
// products are carried) to the correction blocks: it is of the size of the residual, so it
// comes from the accurate products (the Cholesky factor R of X's residual block, or the
// restart coupling) and a correction block's own V^T A Q never overwrites those rows of T.
kl_status run_phase(Eig& E, const Phase& P, int k, int j0, int* restarts, std::vector<double>& theta,
                    std::vector<double>& est, bool* converged) {
    const int b = P.b, m = P.m;
    int j = j0;
    *converged = false;
    theta.assign(m, 0.0);
    est.assign(m, 0.0);
    struct OnePass {
        Eig& e;
        ~OnePass() { e.one_pass = false; }
    } one_pass_guard{E};
    E.one_pass = P.one_pass;
    bool first = true;
    int acc = 0;   // leading basis columns whose products are accurate (correction blocks only)
    for (int it = 0;; ++it) {
        // ---- expansion until the basis is full ----
        bool full = false;
        while (!full) {
            double* Q = E.V() + size_t(j - b) * E.N;
            const bool corr = !first && P.prec_next != P.prec;
            KL_TRY(E.apply(corr ? P.prec_next : P.prec, Q, E.W(), b));
            first = false;
            // keep the raw products: A V[:, j-b:j]
            if (P.carry) {
                cudaError_t ec = launch_copy_block(E.W(), E.N, E.AV() + size_t(j - b) * E.N, E.N, E.N, b, E.s);
                if (ec != cudaSuccess) return cuda_fail(ec, "copy products");
            }
            KL_TRY(E.orthogonalize(E.W(), b, j));
            // T[r0:j, j-b:j] = H[r0:j] (and its mirror); a correction block leaves the rows of
            // the accurate columns as the accurate products set them
            const int r0 = corr ? acc : 0;
            if (!corr) acc = j;
            cudaError_t e = launch_fill_T_block(E.T(), E.mmax, r0, j - b, E.H() + r0, E.mmax, j - r0, b, true, E.s);
            if (e != cudaSuccess) return cuda_fail(e, "fill T");
            if (j + b > m) {
                full = true;
                break;
            }
            if (P.early_rr && !(P.skip_first_rr && it == 0 && j == j0)) {
                // Rayleigh-Ritz on the current basis, residual block = W (not yet normalised)
                KL_TRY(E.sym_eig(j));
                e = E.gram(E.W(), E.N, b, E.W(), E.N, b, E.G(), b);
                if (e != cudaSuccess) return cuda_fail(e, "gram");
                const int nc = std::min(j, k);
                e = launch_residual_norms(E.G(), b, E.S(), E.mmax, j - b, b, nc, E.Est(), E.s);
                if (e != cudaSuccess) return cuda_fail(e, "residual norms");
                std::vector<double> th(nc), rs(nc);
                KL_TRY(host_wait(E.h, E.s));
                KL_CUDA(cudaMemcpyAsync(th.data(), E.Theta(), nc * sizeof(double), cudaMemcpyDeviceToHost, E.s));
                KL_CUDA(cudaMemcpyAsync(rs.data(), E.Est(), nc * sizeof(double), cudaMemcpyDeviceToHost, E.s));
                KL_CUDA(cudaStreamSynchronize(E.s));
                for (int i = 0; i < nc; ++i)
                    if (!std::isfinite(th[i]) || !std::isfinite(rs[i]))
                        return fail(KL_ERR_NUMERIC, "non-finite Ritz values (NaN or Inf in the start block or the operator)");
                bool ok = (nc == k);
                for (int i = 0; i < nc && ok; ++i) ok = rs[i] <= P.tol * fabs(th[i]);
                if (ok) {
                    // Ritz vectors into V[:, 0:ke]
                    const int ke = std::min(std::max(k, P.exit_vecs), j);
                    e = E.gemm(1.0, E.V(), E.N, j, E.S(), E.mmax, ke, 0.0, E.Y(), E.N);
                    if (e != cudaSuccess) return cuda_fail(e, "ritz vectors");
                    e = launch_copy_block(E.Y(), E.N, E.V(), E.N, E.N, ke, E.s);
                    if (e != cudaSuccess) return cuda_fail(e, "copy");
                    if (P.carry) KL_TRY(E.rotate_products(j, ke));
                    for (int i = 0; i < k; ++i) {
                        theta[i] = th[i];
                        est[i] = rs[i];
                    }
                    *converged = true;
                    E.exit_j = j;
                    E.exit_acc = acc;
                    E.exit_restarted = it > 0;
                    return KL_OK;
                }
            }
            bool def = false;
            double* dst = E.V() + size_t(j) * E.N;
            KL_TRY(E.cholqr(E.W(), b, dst, &def));
            if (def) {
                KL_TRY(E.random_orthonormal(dst, b, j));
                // coupling is lost: the new block is a fresh direction (R = 0)
                e = cudaMemsetAsync(E.R(), 0, sizeof(double) * b * b, E.s);
                if (e != cudaSuccess) return cuda_fail(e, "memset");
            }
            // T[j:j+b, j-b:j] = R ; symmetric
            e = launch_fill_T_block(E.T(), E.mmax, j, j - b, E.R(), b, b, b, true, E.s);
            if (e != cudaSuccess) return cuda_fail(e, "fill T");
            j += b;
        }
        // ---- Rayleigh-Ritz on the full basis ----
        KL_TRY(E.sym_eig(j));
        cudaError_t e = E.gram(E.W(), E.N, b, E.W(), E.N, b, E.G(), b);
        if (e != cudaSuccess) return cuda_fail(e, "gram");
        const int nk = std::min(P.keep, j);
        e = launch_residual_norms(E.G(), b, E.S(), E.mmax, j - b, b, nk, E.Est(), E.s);
        if (e != cudaSuccess) return cuda_fail(e, "residual norms");
        KL_TRY(host_wait(E.h, E.s));
        KL_CUDA(cudaMemcpyAsync(theta.data(), E.Theta(), j * sizeof(double), cudaMemcpyDeviceToHost, E.s));
        KL_CUDA(cudaMemcpyAsync(est.data(), E.Est(), nk * sizeof(double), cudaMemcpyDeviceToHost, E.s));
        KL_CUDA(cudaStreamSynchronize(E.s));
        for (int i = 0; i < std::min(k, nk); ++i)
            if (!std::isfinite(theta[i]) || !std::isfinite(est[i]))
                return fail(KL_ERR_NUMERIC, "non-finite Ritz values (NaN or Inf in the start block or the operator)");
        bool ok = true;
        for (int i = 0; i < k; ++i) ok = ok && (est[i] <= P.tol * fabs(theta[i]));
        const bool last = (it >= P.maxrestart);
        const int keep = ok || last ? std::min(std::max(k, P.exit_vecs), j) : P.keep;
        // Ritz vectors V S[:, 0:keep] -> Y -> V[:, 0:keep]
        e = E.gemm(1.0, E.V(), E.N, j, E.S(), E.mmax, keep, 0.0, E.Y(), E.N);
        if (e != cudaSuccess) return cuda_fail(e, "ritz vectors");
        e = launch_copy_block(E.Y(), E.N, E.V(), E.N, E.N, keep, E.s);
        if (e != cudaSuccess) return cuda_fail(e, "copy");
        if (P.carry) KL_TRY(E.rotate_products(j, keep));
        if (!(ok || last) && P.carry && P.prec_next != P.prec && keep <= b) {
            // a restart of a pass with correction blocks: the kept Ritz vectors' products now
            // carry this cycle's correction error (the correction columns acc:j are untouched by
            // the rotation, which rewrote columns 0:keep)
            std::vector<double> ce;
            KL_TRY(E.correction_error(acc, j, keep, &ce));
            E.contam += *std::max_element(ce.begin(), ce.end());
        }
        if (ok || last) {
            *converged = ok;
            E.exit_j = j;
            E.exit_acc = acc;
            E.exit_restarted = it > 0;
            return KL_OK;
        }
        ++*restarts;
        // residual block F = W -> orthonormal block after the kept Ritz vectors
        bool def = false;
        double* dst = E.V() + size_t(keep) * E.N;
        KL_TRY(E.orthogonalize(E.W(), b, keep));   // F is orthogonal to V already; cleans round-off
        KL_TRY(E.cholqr(E.W(), b, dst, &def));
        if (def) {
            KL_TRY(E.random_orthonormal(dst, b, keep));
            e = cudaMemsetAsync(E.R(), 0, sizeof(double) * b * b, E.s);
            if (e != cudaSuccess) return cuda_fail(e, "memset");
        }
        e = launch_set_restart_T(E.T(), E.mmax, E.mmax, E.Theta(), keep, E.R(), b, E.S(), E.mmax, j - b, b, E.s);
        if (e != cudaSuccess) return cuda_fail(e, "restart T");
        j = keep + b;
        acc = keep;   // the kept Ritz vectors carry their products; the coupling is set above
    }
}

// Block LOBPCG (Knyazev's locally optimal block preconditioned conjugate gradient, without a
// preconditioner) for the nx largest eigenpairs, in the orthonormal-basis form: every step
// applies the operator to the residual block R = A X - X Theta only, and Rayleigh-Ritz runs on
// span[X, P, R] (P: the previous step's search directions), kept orthonormal in float64 (CGS2 and
// CholQR2) together with their operator products, so no product is recomputed.
// Basis layout: X in V[:, 0:nx], P in V[:, nx:2nx] (once it exists), R after them; the products
// alike in AV.  On entry V[:, 0:nx] holds an orthonormal start block; with `have_ax` AV[:, 0:nx]
// already holds its products and Theta its Ritz values (a previous phase).  On exit V[:, 0:nx]
// holds the Ritz vectors (descending), AV their products, theta/est the values and the residual
// norms of the k wanted pairs.
kl_status run_lobpcg(Eig& E, int prec, int nx, int k, double tol, int maxit, bool have_ax, int* iters,
                     std::vector<double>& theta, std::vector<double>& est, bool* converged) {
    const int64_t N = E.N;
    double* V = E.V();
    double* AV = E.AV();
    cudaError_t e;
    *converged = false;
    theta.assign(3 * nx, 0.0);
    est.assign(nx, 0.0);
    if (!have_ax) {
        // products of the start block and Rayleigh-Ritz on it
        KL_TRY(E.apply(prec, V, AV, nx));
        e = launch_gram(V, N, nx, AV, N, nx, N, E.T(), E.mmax, E.Part(), E.maxparts, E.s);
        if (e != cudaSuccess) return cuda_fail(e, "gram");
        KL_TRY(E.sym_eig(nx));
        e = launch_gemm_tall(1.0, V, N, N, nx, E.S(), E.mmax, nx, 0.0, E.Y(), N, E.s);
        if (e == cudaSuccess) e = launch_gemm_tall(1.0, AV, N, N, nx, E.S(), E.mmax, nx, 0.0, E.Y2(), N, E.s);
        if (e == cudaSuccess) e = launch_copy_block(E.Y(), N, V, N, N, nx, E.s);
        if (e == cudaSuccess) e = launch_copy_block(E.Y2(), N, AV, N, N, nx, E.s);
        if (e != cudaSuccess) return cuda_fail(e, "ritz block");
    }
    int np = 0;   // columns of P
    for (int it = 0;; ++it) {
        // ---- convergence of the k wanted pairs ----
        e = launch_ritz_resid(AV, V, N, N, nx, E.Theta(), E.Part(), E.maxparts, E.Est(), E.s);
        if (e != cudaSuccess) return cuda_fail(e, "ritz residuals");
        KL_TRY(host_wait(E.h, E.s));
        KL_CUDA(cudaMemcpyAsync(theta.data(), E.Theta(), nx * sizeof(double), cudaMemcpyDeviceToHost, E.s));
        KL_CUDA(cudaMemcpyAsync(est.data(), E.Est(), nx * sizeof(double), cudaMemcpyDeviceToHost, E.s));
        KL_CUDA(cudaStreamSynchronize(E.s));
        bool ok = true;
        for (int i = 0; i < k; ++i) {
            if (!std::isfinite(theta[i]) || !std::isfinite(est[i]))
                return fail(KL_ERR_NUMERIC, "non-finite Ritz values (NaN or Inf in the start block or the operator)");
            est[i] *= fabs(theta[i]);   // launch_ritz_resid gives ||A~'x - theta x|| / |theta|
            ok = ok && est[i] <= tol * fabs(theta[i]);
        }
        *iters = it;
        if (ok || it >= maxit) {
            *converged = ok;
            return KL_OK;
        }
        // ---- residual block, orthonormal against [X, P], and its products ----
        const int r0 = nx + np;
        e = launch_ritz_residual_block(AV, V, N, N, nx, E.Theta(), E.W(), N, E.s);
        if (e != cudaSuccess) return cuda_fail(e, "residual block");
        KL_TRY(E.orthogonalize(E.W(), nx, r0));
        bool def = false;
        KL_TRY(E.cholqr(E.W(), nx, V + size_t(r0) * N, &def));
        if (def) KL_TRY(E.random_orthonormal(V + size_t(r0) * N, nx, r0));
        KL_TRY(E.apply(prec, V + size_t(r0) * N, AV + size_t(r0) * N, nx));
        // ---- Rayleigh-Ritz on Z = [X, P, R] ----
        const int mz = r0 + nx;
        e = launch_gram(V, N, mz, AV, N, mz, N, E.T(), E.mmax, E.Part(), E.maxparts, E.s);
        if (e != cudaSuccess) return cuda_fail(e, "gram");
        KL_TRY(E.sym_eig(mz));
        // new X = Z S[:, 0:nx]; new P = [P, R] S[nx:mz, 0:nx] (the X components dropped); the
        // products alike.  P goes to the spare columns [mz, mz + nx) first.
        double* Pn = V + size_t(mz) * N;
        double* APn = AV + size_t(mz) * N;
        const double* Sx = E.S() + nx;   // rows nx.. of S (column-major, ld mmax)
        e = launch_gemm_tall(1.0, V + size_t(nx) * N, N, N, mz - nx, Sx, E.mmax, nx, 0.0, Pn, N, E.s);
        if (e == cudaSuccess)
            e = launch_gemm_tall(1.0, AV + size_t(nx) * N, N, N, mz - nx, Sx, E.mmax, nx, 0.0, APn, N, E.s);
        if (e == cudaSuccess) e = launch_gemm_tall(1.0, V, N, N, mz, E.S(), E.mmax, nx, 0.0, E.Y(), N, E.s);
        if (e == cudaSuccess) e = launch_gemm_tall(1.0, AV, N, N, mz, E.S(), E.mmax, nx, 0.0, E.Y2(), N, E.s);
        if (e == cudaSuccess) e = launch_copy_block(E.Y(), N, V, N, N, nx, E.s);
        if (e == cudaSuccess) e = launch_copy_block(E.Y2(), N, AV, N, N, nx, E.s);
        if (e == cudaSuccess) e = launch_copy_block(Pn, N, V + size_t(nx) * N, N, N, nx, E.s);
        if (e == cudaSuccess) e = launch_copy_block(APn, N, AV + size_t(nx) * N, N, N, nx, E.s);
        if (e != cudaSuccess) return cuda_fail(e, "lobpcg update");
        // ---- X orthonormal again (the rotations' rounding would otherwise accumulate over the
        // steps), then P orthonormal against X; their products follow every transformation ----
        bool xdef = false;
        KL_TRY(E.cholqr_pair(V, AV, nx, V, AV, &xdef));
        if (xdef) return fail(KL_ERR_NUMERIC, "LOBPCG: the Ritz block lost rank");
        double* P = V + size_t(nx) * N;
        double* AP = AV + size_t(nx) * N;
        KL_TRY(E.orthogonalize(P, nx, nx));                       // P -= X H (twice), H accumulated
        e = launch_gemm_tall(-1.0, AV, N, N, nx, E.H(), E.mmax, nx, 1.0, AP, N, E.s);
        if (e != cudaSuccess) return cuda_fail(e, "lobpcg products");
        bool pdef = false;
        KL_TRY(E.cholqr_pair(P, AP, nx, P, AP, &pdef));
        np = pdef ? 0 : nx;
    }
}

}  // namespace

// outputs of a solve: eigenvalues, residuals (re-measured with the products carried with the
// basis, or a fresh float64 application), eigenvectors, statistics and stage-5 event timing
static kl_status finish_eigs(kl_handle h, Eig& E, const kl_eig_opts& o, int k, double tol, const std::vector<double>& theta,
                      const std::vector<double>& est, int restarts, double ms32, double* evals_host, double* evecs_dev,
                      int64_t ldv, kl_eig_info* info, cudaStream_t s,
                      std::chrono::steady_clock::time_point t0) {
    const int64_t N = h->N;
    cudaError_t e;
    // a bounded wait that gave up inside a tensor-core kernel invalidates the solve
    if (o.precision == KL_P_TC64 || o.precision == KL_P_TC32) KL_TRY(check_device_status(h, s));

    // ---- outputs ----
    for (int i = 0; i < k; ++i) evals_host[i] = theta[i];
    std::vector<double> resid(k, 0.0);
    for (int i = 0; i < k; ++i) resid[i] = est[i] / std::max(fabs(theta[i]), 1e-300);
    if (o.verify) {
        // explicit float64 residuals ||A y - theta y|| / |theta|
        // verify 1: A~'y from the operator products kept with the basis (AV S);
        // verify 2: a fresh application with the float64 kernel
        const double* AY = E.AV();
        if (o.verify == 2) {
            KL_TRY(E.apply(KL_P_FP64, E.V(), E.Y(), k));
            AY = E.Y();
        }
        KL_CUDA(cudaMemcpyAsync(E.Theta(), theta.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
        e = launch_ritz_resid(AY, E.V(), N, N, k, E.Theta(), E.Part(), E.maxparts, E.Est(), s);
        if (e != cudaSuccess) return cuda_fail(e, "ritz residuals");
        KL_TRY(host_wait(h, s));
        KL_CUDA(cudaMemcpyAsync(resid.data(), E.Est(), k * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    if (evecs_dev) {
        e = launch_copy_block(E.V(), N, evecs_dev, ldv, N, k, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy eigenvectors");
    }
    KL_CUDA(cudaStreamSynchronize(s));
    int nconv = 0;
    for (int i = 0; i < k; ++i) nconv += (resid[i] <= tol) ? 1 : 0;
    if (info) {
        info->applies = E.applies;
        info->applies_fp64 = E.applies64;
        info->applies_df64 = E.appliesdf;
        info->applies_tc64 = E.appliestc64;
        info->applies_tc32 = E.appliestc32;
        info->block_applies = E.block_applies;
        info->restarts = restarts;
        info->converged = nconv;
        for (int i = 0; i < 64; ++i) info->resid[i] = i < k ? resid[i] : 0.0;
        info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        info->ms_fp32_phase = ms32;
        info->stage5_calls_fp64 = info->stage5_calls_fp32 = info->stage5_calls_df64 = 0;
        info->ms_stage5_fp64 = info->ms_stage5_fp32 = info->ms_stage5_df64 = 0.0;
        info->pairs_fp64 = info->pairs_fp32 = info->pairs_df64 = 0.0;
        info->stage5_calls_tc64 = info->stage5_calls_tc32 = 0;
        info->ms_stage5_tc64 = info->pairs_tc64 = info->ms_stage5_tc32 = info->pairs_tc32 = 0.0;
        const double pairs = double(h->Nt) * double(h->Nt);
        for (const auto& r : h->prof_rec) {
            float ms = 0.f;
            KL_CUDA(cudaEventElapsedTime(&ms, h->prof_ev[r.ev], h->prof_ev[r.ev + 1]));
            if (r.kind == KL_P_FP64) {
                info->stage5_calls_fp64 += 1;
                info->ms_stage5_fp64 += ms;
                info->pairs_fp64 += pairs;
            } else if (r.kind == KL_P_DF64) {
                info->stage5_calls_df64 += 1;
                info->ms_stage5_df64 += ms;
                info->pairs_df64 += pairs;
            } else if (r.kind == KL_P_TC64) {
                info->stage5_calls_tc64 += 1;
                info->ms_stage5_tc64 += ms;
                info->pairs_tc64 += pairs;
            } else if (r.kind == KL_P_TC32) {
                info->stage5_calls_tc32 += 1;
                info->ms_stage5_tc32 += ms;
                info->pairs_tc32 += pairs;
            } else {
                info->stage5_calls_fp32 += 1;
                info->ms_stage5_fp32 += ms;
                info->pairs_fp32 += pairs;
            }
        }
    }
    if (nconv < k) return fail(KL_ERR_NOT_CONVERGED, "not every wanted eigenpair reached the tolerance");
    return KL_OK;
}

// Block LOBPCG solve (opts.method 2: every application in opts.precision; method 3: a first
// phase with the float32-class operator to tol_low, then the float64-class operator from the
// float32 Ritz block, whose products are recomputed and whose search directions restart).
static kl_status lobpcg_impl(kl_handle h, int k, double tol, const kl_eig_opts& o, double* evals_host, double* evecs_dev,
                      int64_t ldv, kl_eig_info* info, cudaStream_t s, std::chrono::steady_clock::time_point t0) {
    const int64_t N = h->N;
    if (o.precision != KL_P_FP64 && o.precision != KL_P_DF64 && o.precision != KL_P_TC64)
        return fail(KL_ERR_INVALID_ARG, "LOBPCG: opts.precision must be KL_P_FP64, KL_P_DF64 or KL_P_TC64");
    const int nx = o.block >= k ? o.block : std::max(k, int(std::min<int64_t>(32, N / 3)));
    if (nx > 48) return fail(KL_ERR_INVALID_ARG, "LOBPCG: block above 48");
    if (int64_t(3) * nx > N) return fail(KL_ERR_INVALID_ARG, "LOBPCG: 3 x block exceeds the problem dimension");
    const int maxit = o.maxiter > 0 ? o.maxiter : 1000;
    h->prof_on = (info != nullptr);
    h->prof_rec.clear();
    struct ProfOff {
        kl_handle h;
        ~ProfOff() { h->prof_on = false; }
    } prof_off{h};
    Eig E;
    E.h = h;
    E.s = s;
    E.N = N;
    E.seed = o.seed;
    KL_TRY(E.alloc(3 * nx, nx));
    cudaError_t e;
    if (o.start_dev) {
        e = launch_copy_block(o.start_dev, N, E.W(), N, N, nx, s);
        if (e == cudaSuccess) e = launch_gram(E.W(), N, nx, E.W(), N, nx, N, E.G(), nx, E.Part(), E.maxparts, s);
        if (e != cudaSuccess) return cuda_fail(e, "start block");
        std::vector<double> g(size_t(nx) * nx);
        KL_TRY(host_wait(h, s));
        KL_CUDA(cudaMemcpyAsync(g.data(), E.G(), g.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        KL_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nx; ++i)
            if (!std::isfinite(g[size_t(i) * nx + i])) return fail(KL_ERR_NUMERIC, "the start block contains NaN or Inf");
    } else {
        e = launch_random_block(E.W(), N, N, nx, o.seed, 0, s);
        E.rng_offset = uint64_t(N) * nx;
        if (e != cudaSuccess) return cuda_fail(e, "start block");
    }
    bool def = false;
    KL_TRY(E.cholqr(E.W(), nx, E.V(), &def));
    if (def) KL_TRY(E.random_orthonormal(E.V(), nx, 0));
    std::vector<double> theta, est;
    int iters = 0, iters2 = 0;
    bool conv = false;
    double ms32 = 0.0;
    if (o.method == 2) {
        KL_TRY(run_lobpcg(E, o.precision, nx, k, tol, maxit, false, &iters, theta, est, &conv));
    } else {
        const double tl = o.tol_low > 0.0 ? o.tol_low : (o.precision == KL_P_TC64 ? 1e-6 : 1e-5);
        const int lowp = (o.low_precision == KL_P_TC32) ? KL_P_TC32 : KL_P_FP32;
        KL_TRY(run_lobpcg(E, lowp, nx, k, std::max(tl, tol), maxit, false, &iters, theta, est, &conv));
        if (lowp == KL_P_TC32) KL_TRY(check_device_status(h, s));
        KL_CUDA(cudaStreamSynchronize(s));
        ms32 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        // the float32 Ritz block, re-orthonormalised in float64, restarts the iteration with the
        // float64-class operator (its products are recomputed there)
        bool defp = false;
        KL_TRY(E.cholqr(E.V(), nx, E.W(), &defp));
        e = launch_copy_block(E.W(), N, E.V(), N, N, nx, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy");
        KL_TRY(run_lobpcg(E, o.precision, nx, k, tol, maxit, false, &iters2, theta, est, &conv));
    }
    if (o.precision == KL_P_TC64) KL_TRY(check_device_status(h, s));
    return finish_eigs(h, E, o, k, tol, theta, est, iters + iters2, ms32, evals_host, evecs_dev, ldv, info, s, t0);
}

kl_status eigs_impl(kl_handle h, int k, double tol, const kl_eig_opts* opts_in, double* evals_host, double* evecs_dev,
                    int64_t ldv, kl_eig_info* info, cudaStream_t s) {
    auto t0 = std::chrono::steady_clock::now();
    kl_eig_opts o{};
    o.method = 0;
    o.block = 1;
    o.ncv = 0;
    o.maxiter = 0;
    o.seed = 1;
    o.start_dev = nullptr;
    o.tol_low = 0.0;
    o.verify = 1;
    o.precision = KL_P_FP64;
    o.polish_block = 0;
    o.polish_ncv = 0;
    o.low_precision = KL_P_FP32;
    o.nstart = 0;
    if (opts_in) o = *opts_in;
    if (o.method < 0 || o.method > 3) return fail(KL_ERR_INVALID_ARG, "method must be 0, 1, 2 or 3");
    if (o.method >= 2) return lobpcg_impl(h, k, tol, o, evals_host, evecs_dev, ldv, info, s, t0);
    // float32-class arithmetic throughout is allowed for the plain method (results accurate to
    // the float32 operator: residual tolerances of about 1e-5 and above, e.g. training data)
    const bool f32_plain = (o.method == 0 && (o.precision == KL_P_FP32 || o.precision == KL_P_TC32));
    if (o.precision != KL_P_FP64 && o.precision != KL_P_DF64 && o.precision != KL_P_TC64 && !f32_plain)
        return fail(KL_ERR_INVALID_ARG,
                    "opts.precision must be KL_P_FP64, KL_P_DF64 or KL_P_TC64 (or KL_P_FP32 / KL_P_TC32 with method 0)");
    const int b = std::max(1, o.block);
    if (b > 64) return fail(KL_ERR_INVALID_ARG, "block size above 64");
    const int64_t N = h->N;
    int m = o.ncv > 0 ? o.ncv : std::max(2 * k + 1, k + 3 * b);
    m = (m + b - 1) / b * b;
    if (m > 160) m = 160 / b * b;
    if (m < k + 2 * b) return fail(KL_ERR_INVALID_ARG, "basis size too small for k and the block size (need ncv >= k + 2 block, <= 160)");
    if (m > N) return fail(KL_ERR_INVALID_ARG, "basis size exceeds the problem dimension; use a smaller ncv / block");
    const int maxrestart = o.maxiter > 0 ? o.maxiter : 1000;
    // kept Ritz vectors: m - c b with c ~ (m - k) / (2b), at least k
    int c = std::max(1, (m - k) / (2 * b));
    int keep = m - c * b;
    if (keep < k) keep = k;
    while ((m - keep) % b != 0) --keep;

    // float64 polish of the mixed method: one wide block over the kept float32 Ritz vectors
    // a tensor-core float64-class launch costs the same for any width up to 32 vectors (the
    // kernel values, which dominate, are shared by the block), so its polish block defaults to
    // 32 with the vectors beyond k as guards; the other precisions default to k
    const int pol_def = (o.precision == KL_P_TC64) ? std::max(k, int(std::min<int64_t>(32, N / 3))) : k;
    const int pol_b = std::min(std::max(o.polish_block > 0 ? o.polish_block : pol_def, k), 48);
    // polish basis: three blocks when every block takes the accurate arithmetic; four when only
    // the first does (a further correction block costs a float32 application)
    int pol_m = o.polish_ncv > 0 ? o.polish_ncv / pol_b * pol_b : (o.polish_accurate ? 3 : 4) * pol_b;
    pol_m = std::min(std::max(pol_m, 2 * pol_b), 160 / pol_b * pol_b);

    // stage-5 event timing for the whole call (read back at the end)
    h->prof_on = (info != nullptr);
    h->prof_rec.clear();
    struct ProfOff {
        kl_handle h;
        ~ProfOff() { h->prof_on = false; }
    } prof_off{h};

    Eig E;
    E.h = h;
    E.s = s;
    E.N = N;
    E.seed = o.seed;
    // a wider start subspace is compressed to its `b` leading Ritz vectors before the iteration
    const int nst = (o.start_dev && o.nstart > b) ? o.nstart : b;
    if (o.nstart < 0 || nst > 64 || nst > m)
        return fail(KL_ERR_INVALID_ARG, "opts.nstart must lie in block..min(64, basis size)");
    const int cap_m = std::max(m, pol_m), cap_b = std::max(std::max(b, pol_b), nst);
    KL_TRY(E.alloc(cap_m, cap_b));
    cudaError_t e = cudaMemsetAsync(E.T(), 0, sizeof(double) * cap_m * cap_m, s);
    if (e != cudaSuccess) return cuda_fail(e, "memset");

    // ---- start block ----
    if (o.start_dev) {
        // a caller's start block with NaN or Inf is an error, not a rank-deficient block to replace
        e = launch_copy_block(o.start_dev, N, E.W(), N, N, nst, s);
        if (e == cudaSuccess) e = launch_gram(E.W(), N, nst, E.W(), N, nst, N, E.G(), nst, E.Part(), E.maxparts, s);
        if (e != cudaSuccess) return cuda_fail(e, "start block");
        std::vector<double> g(size_t(nst) * nst);
        KL_TRY(host_wait(h, s));
        KL_CUDA(cudaMemcpyAsync(g.data(), E.G(), g.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        KL_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nst; ++i)
            if (!std::isfinite(g[size_t(i) * nst + i]))
                return fail(KL_ERR_NUMERIC, "the start block contains NaN or Inf");
    }
    if (o.start_dev && nst > b) {
        // Rayleigh-Ritz on span(start): orthonormal basis in V[:, 0:nst], its products in AV,
        // T = V^T A V, then W = the b leading Ritz vectors
        e = launch_copy_block(o.start_dev, N, E.W(), N, N, nst, s);
        if (e != cudaSuccess) return cuda_fail(e, "start block");
        bool sdef = false;
        KL_TRY(E.cholqr(E.W(), nst, E.V(), &sdef));
        if (sdef) return fail(KL_ERR_INVALID_ARG, "start columns are numerically rank deficient");
        const int p1 = (o.method == 1) ? ((o.low_precision == KL_P_TC32) ? KL_P_TC32 : KL_P_FP32) : o.precision;
        KL_TRY(E.apply(p1, E.V(), E.AV(), nst));
        e = launch_gram(E.V(), N, nst, E.AV(), N, nst, N, E.T(), E.mmax, E.Part(), E.maxparts, s);
        if (e != cudaSuccess) return cuda_fail(e, "gram");
        KL_TRY(E.sym_eig(nst));
        e = launch_gemm_tall(1.0, E.V(), N, N, nst, E.S(), E.mmax, b, 0.0, E.W(), N, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(E.T(), 0, sizeof(double) * cap_m * cap_m, s);
    } else if (o.start_dev) {
        e = launch_copy_block(o.start_dev, N, E.W(), N, N, b, s);
    } else {
        e = launch_random_block(E.W(), N, N, b, o.seed, 0, s);
        E.rng_offset = uint64_t(N) * b;
    }
    if (e != cudaSuccess) return cuda_fail(e, "start block");
    bool def = false;
    KL_TRY(E.cholqr(E.W(), b, E.V(), &def));
    if (def) KL_TRY(E.random_orthonormal(E.V(), b, 0));

    std::vector<double> theta, est;
    int restarts = 0;
    bool conv = false;
    double ms32 = 0.0;
    if (o.method == 0) {
        Phase P{o.precision, b, m, keep, tol, false, maxrestart, k, o.precision};
        KL_TRY(run_phase(E, P, k, b, &restarts, theta, est, &conv));
    } else {
        // the float32 operator's error is relative to |lambda_1|, the residual test to |theta_i|:
        // before a tensor-core polish (one launch costs as much as ~6 float32 block applications)
        // the float32 phase goes one decade further, which also keeps the correction blocks few
        const double tl = o.tol_low > 0.0 ? o.tol_low : (o.precision == KL_P_TC64 ? 1e-6 : 1e-5);
        const int pb = std::min(pol_b, m);
        const int lowp = (o.low_precision == KL_P_TC32) ? KL_P_TC32 : KL_P_FP32;
        Phase P1{lowp, b, m, keep, std::max(tl, tol), false, maxrestart, pb, lowp};
        P1.carry = false;   // the polish applies the operator to the Ritz block afresh
        P1.one_pass = true;
        KL_TRY(run_phase(E, P1, k, b, &restarts, theta, est, &conv));
        if (lowp == KL_P_TC32) KL_TRY(check_device_status(h, s));
        KL_CUDA(cudaStreamSynchronize(s));
        ms32 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        // polish: V[:, 0:pb] holds the leading float32 Ritz vectors (orthonormal in float64);
        // they form the first, wide block of a float64 block Lanczos run.
        // the correction blocks take the float32 class; blocks wider than 16 vectors run on the
        // tensor-core float32 kernel (one launch for up to 32 vectors, measured 23.1 ms against
        // 2 x 13.6 ms for the CUDA-core kernel's two 16-wide groups at 132,651 points, 2.3 against
        // 2.9 ms at 39,304; for many small instances solved together, 1.53 s against 2.4 s with
        // the CUDA-core kernel's shared launches)
        const int corr_p = (lowp == KL_P_FP32 && pb > 16) ? KL_P_TC32 : lowp;
        Phase P2{o.precision, pb, pol_m, pb, tol, true, maxrestart, pb, o.polish_accurate ? o.precision : corr_p};
        // With float32 correction blocks the residuals carried with the Ritz vectors are off by
        // about eps32 ||A~'|| |s|, s their coefficients on the correction blocks.  Where the
        // float32 phase left a wanted vector far from the float64 one (a pair whose eigenvalue is
        // small against lambda_1 and close to its neighbour's) that can exceed the tolerance:
        // the residuals are then re-measured from the carried products, the bound
        // eps32 ||(A~'Q) s_i|| is estimated from the correction blocks' products and Rayleigh-Ritz
        // coefficients, and a pass whose residuals, or residuals plus that estimate, miss the
        // tolerance starts again from its
        // Ritz vectors with one more accurate application (whose first Rayleigh-Ritz check uses
        // accurate products only; the error a pass leaves shrinks by eps32 ||A~'|| / |theta_k|);
        // after kMaxPolishPasses the correction blocks take the accurate arithmetic as well.
        constexpr int kMaxPolishPasses = 4;

        for (int pass = 0;; ++pass) {
            // re-orthonormalise the Ritz block in float64 (CholQR2) before it becomes the first
            // block of the accurate phase
            {
                bool defp = false;
                KL_TRY(E.cholqr(E.V(), pb, E.W(), &defp));
                e = launch_copy_block(E.W(), N, E.V(), N, N, pb, s);
                if (e != cudaSuccess) return cuda_fail(e, "copy");
            }
            // the active block is V[:, 0:pb]; T is rebuilt by the first expansion
            e = cudaMemsetAsync(E.T(), 0, sizeof(double) * cap_m * cap_m, s);
            if (e != cudaSuccess) return cuda_fail(e, "memset");
            // the float32 Ritz block alone carries residuals of about tol_low: no check before the
            // first correction block unless tol_low is within a decade of tol
            P2.skip_first_rr = (pass == 0 && tl >= 10.0 * tol);
            E.contam = 0.0;
            KL_TRY(run_phase(E, P2, k, pb, &restarts, theta, est, &conv));
            if (!conv || P2.prec_next == P2.prec) break;
            // residuals ||A~'y - theta y|| of the k wanted Ritz vectors from their carried products
            e = launch_ritz_resid(E.AV(), E.V(), N, N, k, E.Theta(), E.Part(), E.maxparts, E.Est(), s);
            if (e != cudaSuccess) return cuda_fail(e, "ritz residuals");
            std::vector<double> rx(k);
            KL_TRY(host_wait(h, s));
            KL_CUDA(cudaMemcpyAsync(rx.data(), E.Est(), k * sizeof(double), cudaMemcpyDeviceToHost, s));
            KL_CUDA(cudaStreamSynchronize(s));
            bool ok = true;   // rx holds ||A~'y - theta y|| / |theta|
            for (int i = 0; i < k; ++i) ok = ok && rx[i] <= tol;
            // those residuals may still be off by the float32 operators' error on the correction
            // blocks' part of the products, about eps32 ||(A~'Q) s_i|| (s_i: the Ritz vector's
            // coefficients on the correction blocks Q); where a residual plus that estimate
            // exceeds the tolerance, one more pass measures the residuals with accurate products
            if (ok) {
                // a pass that restarted kept Ritz vectors whose products carry earlier cycles'
                // corrections, which a float32 phase far from the float64 vectors makes large
                // (measured: 0.3 of the tolerance for lambda_1 / lambda_8 ~ 800): it is verified
                // by another pass; otherwise the last cycle's estimate decides
                bool risky = E.exit_restarted;
                std::vector<double> ce;
                if (!risky) KL_TRY(E.correction_error(E.exit_acc, E.exit_j, k, &ce));
                for (int i = 0; i < k && !risky; ++i) risky = rx[i] + (E.contam + ce[i]) / fabs(theta[i]) > tol;
                if (!risky) break;
            }
            ++restarts;
            if (pass + 1 >= kMaxPolishPasses) P2.prec_next = P2.prec;
        }
    }

    return finish_eigs(h, E, o, k, tol, theta, est, restarts, ms32, evals_host, evecs_dev, ldv, info, s, t0);
}

}  // namespace kl
