// Internal declarations shared by the translation units of libkl.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "kl.h"

namespace kl {

// ----------------------------------------------------------------------------------------
// error handling
// ----------------------------------------------------------------------------------------
void set_error(const std::string& msg);
kl_status fail(kl_status st, const std::string& msg);
const std::string& last_error_message();   // this thread's last message
int num_sms();                             // SMs of the current device (cached)
kl_status cuda_fail(cudaError_t e, const char* what);
void count_launches(int n);   // kernel-launch accounting (kl_kernel_launches)

#define KL_CUDA(...)                                                   \
    do {                                                                \
        cudaError_t e_ = (__VA_ARGS__);                                        \
        if (e_ != cudaSuccess) return ::kl::cuda_fail(e_, #__VA_ARGS__);       \
    } while (0)

#define KL_TRY(...)                                                    \
    do {                                                                \
        kl_status s_ = (__VA_ARGS__);                                          \
        if (s_ != KL_OK) return s_;                                     \
    } while (0)

// ----------------------------------------------------------------------------------------
// host set-up (setup.cpp)
// ----------------------------------------------------------------------------------------
struct Direction {
    int p = 0, ne = 0, pt = 0, net = 0;
    int n = 0, nt = 0;
    std::vector<double> itf;  // patch interfaces (C^0 trial, C^{-1} interpolation space)
    std::vector<double> xi;   // Greville abscissae of the interpolation space (nt)
    std::vector<int> side;    // -1: xi[i] is evaluated from the left (a C^{-1} knot), else 0
    std::vector<double> C;    // C_k = B~_k^{-T} M_k L_k^{-T}, nt x n row-major
    std::vector<double> Linv; // L_k^{-1}, n x n row-major (lower triangular)
    std::vector<double> L;    // L_k, Z_k = L_k L_k^T, n x n row-major (lower triangular)
};

kl_status build_direction(int p, int ne, int pt, int net, const std::vector<double>& interfaces, Direction* out);
kl_status build_prolongation(const Direction& c, const Direction& f, std::vector<double>* Q);

// tensor-product NURBS geometry map: knots per direction, control records (x, y, z, w),
// direction 1 fastest; directions >= dim have one control point
struct NurbsMap {
    int dim = 0;
    int deg[3] = {0, 0, 0};
    int n[3] = {1, 1, 1};
    std::vector<double> knots[3];
    std::vector<double> ctrl;
};
// the map's non-zero basis functions of direction k at one abscissa: span, values, derivatives
// (directions k >= dim: the single function 1)
struct MapBasis1D {
    int span = 0;
    double N[16] = {}, dN[16] = {};
};
void nurbs_basis_1d(const NurbsMap& m, int k, double x, int side, MapBasis1D* out);
// F(xh) and det DF(xh) from the basis values of the three directions at xh (side < 0 in
// nurbs_basis_1d takes the left limit, at a C^0 knot of the map)
void nurbs_map_from_basis(const NurbsMap& m, const MapBasis1D* const b[3], double* X, double* detDF);

// host set-up shared by kl_create and the host-only inspection entry points:
// validate a geometry (for KL_GEOM_NURBS copy its map into *nm), build directions 0..dim-1 of a
// space, and map the Greville grid (X: Ntilde x 3 row-major, direction 1 fastest; J = sqrt(det DF))
kl_status parse_geometry(const kl_geometry* geom, NurbsMap* nm);
kl_status build_space(int dim, const kl_space* space, Direction* dir);
kl_status map_greville_points(const kl_geometry* geom, const NurbsMap& nm, const Direction* dir,
                              std::vector<double>* X, std::vector<double>* J);

// ----------------------------------------------------------------------------------------
// device kernels (launchers)
// ----------------------------------------------------------------------------------------
// Mode-k contraction of a block of nvec tensors viewed as [A][n][B]:
//   Y[v][a][i][b] = sum_j Ct[j * m + i] * X[v][a][j][b] (* scale[a][i][b] if scale != null)
template <typename Tin, typename Tc, typename Tout>
cudaError_t launch_contract(const Tin* X, int64_t ldx, Tout* Y, int64_t ldy, const Tc* Ct, int64_t A,
                            int n, int m, int64_t B, int nvec, const Tc* scale, cudaStream_t s);

struct CovParams {
    int kind;              // kl_kernel_kind
    int poly_m;            // exponent of the polynomial test kernel
    int64_t Nt;            // number of points
    int64_t ldp;           // stride between the x, y, z coordinate arrays
    const double* P64;     // 3 x ldp, coordinates (pre-scaled for EXP/GAUSS/EXP_SEPARABLE)
    const float* P32;      // 3 x ldp, float coordinates pre-scaled for base-2 exponentials
    const double* tab;     // 1024-entry table 2^(j/1024)
    const float* Pdf;      // 6 x ldp: x, y, z heads then tails (double-float coordinates in grid
                           // form: heads on one power-of-two grid q, |tail| <= q/2)
    const float* tabdf;    // 2^(-j/64), j = 0..63: 64 heads then 64 tails
    float gscale = 1.f;    // power of two with gscale * |Gamma| <= 1 (tensor-core float64-class path)
};

// Stage 5: z[:, v] = scale2 * (J .) sum_l Gamma(x_k, x_l) u[:, v]; partial sums over column
// splits go to `part` (splits * nvec * Nt doubles) and are combined in fixed order.
cudaError_t launch_covmv64(const CovParams& cp, const double* U, int64_t ldu, int nvec, double* Z,
                           int64_t ldz, double scale2, const double* J, double* part, int splits,
                           cudaStream_t s);
cudaError_t launch_covmv32(const CovParams& cp, const float* U, int64_t ldu, int nvec, double* Z,
                           int64_t ldz, double scale2, const double* J, double* part, int splits,
                           cudaStream_t s);
int covmv_splits(int64_t Nt, int nvec, bool fp32);
// tensor-core (tcgen05) float32-class stage 5 (exact 3-digit slicing, covmv_tcx.cu) for groups of
// 32 vectors; `part` holds
// covmv_tc_part_doubles doubles, `img` covmv_tc_image_bytes bytes; `status` is a device int that
// a CTA sets to KL_ERR_TIMEOUT when a bounded wait gives up
cudaError_t launch_covmv_tc(const CovParams& cp, const float* U, int64_t ldu, int nvec, double* Z, int64_t ldz,
                            double scale2, const double* J, double* part, void* img, int* status, cudaStream_t s);
size_t covmv_tc_part_doubles(int64_t Nt);
size_t covmv_tc_image_bytes(int64_t Nt);
// tensor-core float64-class stage 5 (exact bfloat16 slicing, see covmv_tcx.cu) for groups of
// 32 vectors; `part` holds covmv_tc64_part_doubles doubles, `img` covmv_tc64_image_bytes bytes
cudaError_t launch_covmv_tc64(const CovParams& cp, const double* U, int64_t ldu, int nvec, double* Z, int64_t ldz,
                              double scale2, const double* J, double* part, void* img, int* status, cudaStream_t s);
size_t covmv_tc64_part_doubles(int64_t Nt);
size_t covmv_tc64_image_bytes(int64_t Nt);
// the symmetric float64-class tensor-core stage 5 (each kernel value serves both pairs; column
// sums added with atomics); used for KL_P_TC64 when tc_symmetric_used(Ntilde)
cudaError_t launch_covmv_tcs64(const CovParams& cp, const double* U, int64_t ldu, int nvec, double* Z, int64_t ldz,
                               double scale2, const double* J, double* part, void* img, int* status, cudaStream_t s);
size_t covmv_tcs64_part_doubles(int64_t Nt);
size_t covmv_tcs64_image_bytes(int64_t Nt);
void set_tc_symmetric(bool on);
bool tc_symmetric_used(int64_t Nt);
// Symmetric stage 5 (each kernel value serves the pairs (k, l) and (l, k)): points are cut into
// T tiles of 256 and every unordered tile pair is evaluated once.  Two schedules:
//   * triangular: one launch, one CTA per pair (I <= J); row sums of pair (I, J) go to partial
//     slot J and column sums to slot I, so T slots of nv x Ntilde doubles are needed;
//   * band (bounded workspace): the pairs {I, (I + d) mod T}, d = 0 .. floor(T/2), taken in
//     launches of W consecutive bands d; CTA (I, s) of a launch takes the W/S bands
//     d0 + s W/S .. and keeps the row sums of tile I in registers across them (row slot s),
//     while each band's column sums go to column slot S + (d - d0).  Within a launch every
//     slot position has one writer; the launches run in order on the stream and add into the
//     slots, which start at zero, so the sum is deterministic with S + W slots whatever Ntilde.
// The band schedule is used when the triangular one would need more than the slot limit
// (set_sym_slot_limit, default 512 MiB).
constexpr int kSymTileSize = 256;
constexpr int kSymBandW = 16, kSymBandS = 4;
struct SymPlan {
    bool band = false;
    int T = 0;          // tiles
    int D = 0;          // bands 0 .. D-1 (D = T/2 + 1)
    int launches = 1;
    int slots = 0;      // partial slots of nv x Ntilde doubles
};
SymPlan sym_plan(int64_t Nt, int nv);
size_t sym_part_doubles(int64_t Nt, int nv);
void set_sym_slot_limit(int64_t bytes);
struct SymBand {        // one launch of the band schedule
    int T, D, d0, nd, S;
};
#ifdef __CUDACC__
// band d (and tile J) of CTA (I, s), step k of a band launch; false when that step has no pair
__device__ __forceinline__ bool sym_band_pair(const SymBand& b, int I, int s, int k, int* J, int* d) {
    const int dd = b.d0 + s * b.nd + k;
    if (dd >= b.D) return false;
    if ((b.T & 1) == 0 && 2 * dd == b.T && I >= b.T / 2) return false;   // {I, I + T/2} once
    *d = dd;
    *J = (I + dd) % b.T;
    return true;
}
#endif

cudaError_t launch_covmv32_sym(const CovParams& cp, const float* U, int64_t ldu, int nvec, double* Z,
                               int64_t ldz, double scale2, const double* J, double* part, int splits,
                               cudaStream_t s);
cudaError_t launch_covmv64_sym(const CovParams& cp, const double* U, int64_t ldu, int nvec, double* Z,
                               int64_t ldz, double scale2, const double* J, double* part, int splits,
                               cudaStream_t s);
cudaError_t launch_covmv_df(const CovParams& cp, const double* U, int64_t ldu, int nvec, double* Z,
                            int64_t ldz, double scale2, const double* J, double* part, int splits,
                            cudaStream_t s);
int covmv_df_splits(int64_t Nt);
size_t covmv_df_part_doubles(int64_t Nt, int nvec);   // flat (non-symmetric) double-float partials

// dense block linear algebra (linalg.cu)
cudaError_t launch_gram(const double* A, int64_t lda, int p, const double* B, int64_t ldb, int q,
                        int64_t N, double* out, int ldo, double* part, int maxparts, cudaStream_t s);
int gram_parts(int64_t N);
cudaError_t launch_gemm_tall(double alpha, const double* A, int64_t lda, int64_t N, int p,
                             const double* B, int ldb, int q, double beta, double* C, int64_t ldc,
                             cudaStream_t s);
// the same two products in double-float arithmetic on the float32 pipe (about 2^-46 of each
// result's magnitude): for phases whose operator is float32-accurate
cudaError_t launch_gram_df(const double* A, int64_t lda, int p, const double* B, int64_t ldb, int q,
                           int64_t N, double* out, int ldo, double* part, int maxparts, cudaStream_t s);
cudaError_t launch_gemm_tall_df(double alpha, const double* A, int64_t lda, int64_t N, int p,
                                const double* B, int ldb, int q, double beta, double* C, int64_t ldc,
                                cudaStream_t s);
cudaError_t launch_chol_inv(double* G, int ldg, int b, double* Rinv, double* R, int* flag,
                            cudaStream_t s);
cudaError_t launch_random_block(double* V, int64_t ldv, int64_t N, int b, uint64_t seed,
                                uint64_t offset, cudaStream_t s);
// Symmetric eigen-decomposition of the m x m (m <= 160) matrix T (column-major, ld ldt) by
// float64 parallel cyclic Jacobi in one CTA: sorted eigenvalues (descending) and eigenvectors S.
// work: m^2 doubles.  The double-float kernel (m <= 112) rotates a pair while its off-diagonal
// entry exceeds off_tol sqrt(|T_aa T_bb|) (1e-14: to double-float accuracy).
cudaError_t launch_sym_eig_ws(const double* T, int ldt, int m, double* evals, double* S, int lds,
                              double* work, int* sweeps_out, cudaStream_t s, float off_tol = 1e-14f);
cudaError_t launch_residual_norms(const double* G, int ldg, const double* S, int lds, int srow0,
                                  int b, int ncols, double* out, cudaStream_t s);
cudaError_t launch_ritz_resid(const double* AY, const double* Y, int64_t ld, int64_t N, int k,
                              const double* theta, double* part, int maxparts, double* out,
                              cudaStream_t s);
cudaError_t launch_set_restart_T(double* T, int ldt, int m, const double* theta, int p,
                                 const double* R, int ldr, const double* S, int lds, int srow0,
                                 int b, cudaStream_t s);
// W[:, c] = AX[:, c] - theta[c] X[:, c] for c < nc (theta on the device)
cudaError_t launch_ritz_residual_block(const double* AX, const double* X, int64_t ld, int64_t N, int nc,
                                      const double* theta, double* W, int64_t ldw, cudaStream_t s);
cudaError_t launch_copy_block(const double* src, int64_t lds, double* dst, int64_t ldd,
                              int64_t rows, int cols, cudaStream_t s);
cudaError_t launch_to_float(const double* src, int64_t lds, float* dst, int64_t ldd, int64_t rows,
                            int cols, cudaStream_t s);
cudaError_t launch_fill_T_block(double* T, int ldt, int r0, int c0, const double* H, int ldh,
                                int rows, int cols, bool symmetric, cudaStream_t s);
cudaError_t launch_add_inplace(double* H, const double* H2, int n, cudaStream_t s);

// ----------------------------------------------------------------------------------------
// handle
// ----------------------------------------------------------------------------------------
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};
kl_status ensure(DevBuf& b, size_t bytes);
void release(DevBuf& b);

}  // namespace kl

namespace kl {
struct BatchRendezvous;
}

struct kl_handle_s {
    int dim = 0;
    kl_kernel kernel{};
    kl::Direction dir[3];
    int n[3] = {1, 1, 1}, nt[3] = {1, 1, 1};
    int64_t N = 0, Nt = 0;
    int64_t ldw = 0;              // leading dimension of the intermediate tensors (largest stage size)
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    float gscale = 1.f;       // see CovParams::gscale
    std::vector<double> X_host;  // Nt x 3 row-major physical points
    std::vector<double> J_host;  // Nt: J = sqrt(det DF) at the Greville points
    kl::BatchRendezvous* batch = nullptr;   // set while kl_eigs_batched solves this instance
    cudaEvent_t batch_ready = nullptr;       // u of this instance is ready for the batched stage 5
    cudaEvent_t host_sync = nullptr;         // blocking-sync event of host_wait inside a batched solve
    // device set-up data
    double* dCt[3] = {nullptr, nullptr, nullptr};   // forward operator of mode k, layout n_k x nt_k
    double* dC[3] = {nullptr, nullptr, nullptr};    // backward operator of mode k, layout nt_k x n_k
    float* fCt[3] = {nullptr, nullptr, nullptr};
    float* fC[3] = {nullptr, nullptr, nullptr};
    double* dLinvT[3] = {nullptr, nullptr, nullptr}; // (L_k^{-T})^T layout for kl_to_bspline
    double* dP = nullptr;     // 3 x Nt pre-scaled coordinates
    float* fP = nullptr;      // 3 x Nt float coordinates scaled for ex2
    double* dJ = nullptr;     // Nt
    float* fJ = nullptr;      // Nt
    double* dTab = nullptr;   // 1024: 2^(j/1024) for the float64 exponential
    float* dfP = nullptr;     // 6 x Nt double-float coordinates (pre-scaled like dP)
    float* dfTab = nullptr;   // 128: double-float 2^(-j/64)
    int* dStatus = nullptr;   // device status word of the kernels with bounded waits (0 = ok)
    // workspace
    kl::DevBuf w_a, w_b, w_f32a, w_f32b, w_part, w_tcimg;
    // stage-5 event timing (enabled by kl_eigs while it runs)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;       // pool, two per record
    struct ProfRec { int ev; int kind; int nvec; };   // kind: kl_precision
    std::vector<ProfRec> prof_rec;
};

namespace kl {
kl_status apply_impl(kl_handle h, int precision, const double* v, int64_t ldv, double* y,
                     int64_t ldy, int nvec, cudaStream_t s);
kl_status forward_impl(kl_handle h, const double* v, int64_t ldv, double* u, int64_t ldu, int nvec,
                       cudaStream_t s);
kl_status covmv_impl(kl_handle h, int precision, const double* u, int64_t ldu, double* z,
                     int64_t ldz, int nvec, bool withJ, cudaStream_t s);
kl_status backward_impl(kl_handle h, const double* z, int64_t ldz, double* y, int64_t ldy,
                        int nvec, bool zHasJ, cudaStream_t s);
kl_status check_device_status(kl_handle h, cudaStream_t s);
// Called before a synchronous device-to-host read on `s`.  Inside kl_eigs_batched (one host
// thread per instance, usually more threads than cores) it returns once `s` has drained, the
// thread asleep on a blocking-sync event rather than spinning, so that the instances with work
// to issue get the cores; otherwise it does nothing and the read itself waits (spinning: the
// lowest latency for a lone solve).
kl_status host_wait(kl_handle h, cudaStream_t s);
kl_status eigs_impl(kl_handle h, int k, double tol, const kl_eig_opts* opts, double* evals_host,
                    double* evecs_dev, int64_t ldv, kl_eig_info* info, cudaStream_t s);

CovParams cov_params_of(kl_handle h);
// one application split into its stages (the batched path joins other instances at stage 5)
struct ApplyBufs {
    const void* u = nullptr;   // stage-4 output: double, or float for the float32 paths
    double* z = nullptr;       // stage-5 output
    int64_t ld = 0;
};
kl_status apply_forward(kl_handle h, int precision, const double* v, int64_t ldv, int nvec, cudaStream_t s,
                        ApplyBufs* b);
kl_status apply_backward(kl_handle h, int precision, const ApplyBufs& b, double* y, int64_t ldy, int nvec,
                         cudaStream_t s);
// batched stage 5 (batch.cu)
kl_status batch_stage5(kl_handle h, int prec, const void* U, int64_t ldu, double* Z, int64_t ldz, int nv,
                       bool withJ, cudaStream_t s);
}  // namespace kl
