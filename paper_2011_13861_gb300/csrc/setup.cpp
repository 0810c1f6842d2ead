// Host set-up of the univariate factors (float64, once per handle).
//
// For one parametric direction this builds, from the degree and the number of uniform
// elements of the trial space (B-splines B_i, Sec. 2.3) and of the interpolation space
// (B~_i, Sec. 4.2):
//   Z_k   = int B_i B_j            Gauss-Legendre, p+1 points per element (Sec. 3.5 Remark)
//   L_k   with Z_k = L_k L_k^T     (Sec. 4.1, eq. cholesky)
//   M_k   = int B~_i B_j           Gauss-Legendre on the merged breakpoints (Sec. 4.3)
//   B~_k  = B~_j(xi_i)             collocation at the Greville abscissae (Sec. 4.2)
// and folds them into the single dense factor used by the device contractions,
//   C_k = B~_k^{-T} M_k L_k^{-T}   (n~_k x n_k),
// so that the operator of Sec. 4.4.1 reads A~' = C^T J Gamma J C with C = C_d (x) ... (x) C_1.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kl_internal.h"

namespace kl {
namespace {

std::vector<double> open_knots(int p, int ne) {
    std::vector<double> t;
    for (int i = 0; i <= p; ++i) t.push_back(0.0);
    for (int i = 1; i < ne; ++i) t.push_back(double(i) / double(ne));
    for (int i = 0; i <= p; ++i) t.push_back(1.0);
    return t;
}

// Knot span s with t[s] <= x < t[s+1], clamped to the last non-empty span at x = t.back().
int find_span(const std::vector<double>& t, int p, double x) {
    int n = int(t.size()) - p - 1;
    if (x >= t[n]) return n - 1;
    if (x <= t[p]) return p;
    int lo = p, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (x < t[mid]) hi = mid; else lo = mid;
    }
    return lo;
}

// Span s with t[s] < x <= t[s+1] (the left limit at a knot x), clamped to the first non-empty span.
int find_span_left(const std::vector<double>& t, int p, double x) {
    int s = find_span(t, p, x);
    while (s > p && t[size_t(s)] >= x) --s;
    return s;
}

// The p+1 non-zero B-splines N_{s-p..s}(x) on span s, by the triangular scheme of
// "left"/"right" knot distances (de Boor's recurrence written per span).
void nonzero_basis(const std::vector<double>& t, int p, int s, double x, double* N) {
    std::vector<double> left(p + 1), right(p + 1);
    N[0] = 1.0;
    for (int j = 1; j <= p; ++j) {
        left[j] = x - t[s + 1 - j];
        right[j] = t[s + j] - x;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            double denom = right[r + 1] + left[j - r];
            double temp = denom != 0.0 ? N[r] / denom : 0.0;
            N[r] = saved + right[r + 1] * temp;
            saved = left[j - r] * temp;
        }
        N[j] = saved;
    }
}

// Derivatives of the p+1 non-zero B-splines N_{s-p..s} at x from the degree p-1 functions
// of the same span: d/dx N_{i,p} = p N_{i,p-1}/(t_{i+p} - t_i) - p N_{i+1,p-1}/(t_{i+p+1} - t_{i+1}).
void nonzero_basis_derivative(const std::vector<double>& t, int p, int s, double x, double* dN) {
    if (p == 0) {
        dN[0] = 0.0;
        return;
    }
    std::vector<double> Nm(p);
    nonzero_basis(t, p - 1, s, x, Nm.data());   // N_{s-p+1..s, p-1}
    for (int r = 0; r <= p; ++r) {
        const int i = s - p + r;
        double v = 0.0;
        if (r >= 1) {
            const double den = t[i + p] - t[i];
            if (den > 0.0) v += p * Nm[r - 1] / den;
        }
        if (r <= p - 1) {
            const double den = t[i + p + 1] - t[i + 1];
            if (den > 0.0) v -= p * Nm[r] / den;
        }
        dN[r] = v;
    }
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_q (three-term recurrence).
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (q + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= q; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = q * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // refresh the derivative at the converged node
        {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= q; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = q * (z * p0 - p1) / (z * z - 1.0);
        }
        x[i] = -z;
        x[q - 1 - i] = z;
        w[i] = w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// G[i][j] += weight * Na[i] * Nb[j] over the non-zero functions of two spaces at x.
struct Space {
    std::vector<double> t;
    int p;
    int n;
};

Space make_space(int p, int ne) {
    Space s;
    s.t = open_knots(p, ne);
    s.p = p;
    s.n = ne + p;
    return s;
}

// open uniform knots with every interface (an interior breakpoint j / ne) raised to multiplicity
// `mult`; false if a value is not such a breakpoint
bool make_space_itf(int p, int ne, const std::vector<double>& itf, int mult, Space* out) {
    Space s = make_space(p, ne);
    for (double x : itf) {
        const double j = std::round(x * ne);
        if (!(j > 0.0 && j < double(ne)) || std::fabs(x * ne - j) > 1e-12) return false;
        const double xv = j / double(ne);
        int have = 0;
        for (double y : s.t) have += (y == xv);
        for (int r = have; r < mult; ++r) s.t.push_back(xv);
    }
    std::sort(s.t.begin(), s.t.end());
    s.n = int(s.t.size()) - p - 1;
    *out = s;
    return true;
}

// int_0^1 Ba_i Bb_j over the union of the breakpoints of both spaces, q Gauss points each.
std::vector<double> cross_mass(const Space& a, const Space& b, int q) {
    std::vector<double> br(a.t);
    br.insert(br.end(), b.t.begin(), b.t.end());
    std::sort(br.begin(), br.end());
    br.erase(std::unique(br.begin(), br.end()), br.end());
    std::vector<double> gx, gw;
    gauss_legendre(q, gx, gw);
    std::vector<double> G(size_t(a.n) * b.n, 0.0);
    std::vector<double> Na(a.p + 1), Nb(b.p + 1);
    for (size_t e = 0; e + 1 < br.size(); ++e) {
        double x0 = br[e], x1 = br[e + 1], h = x1 - x0;
        double mid = 0.5 * (x0 + x1);
        int sa = find_span(a.t, a.p, mid), sb = find_span(b.t, b.p, mid);
        for (int g = 0; g < q; ++g) {
            double x = mid + 0.5 * h * gx[g], wt = 0.5 * h * gw[g];
            nonzero_basis(a.t, a.p, sa, x, Na.data());
            nonzero_basis(b.t, b.p, sb, x, Nb.data());
            for (int i = 0; i <= a.p; ++i)
                for (int j = 0; j <= b.p; ++j)
                    G[size_t(sa - a.p + i) * b.n + (sb - b.p + j)] += wt * Na[i] * Nb[j];
        }
    }
    return G;
}

// In-place inverse of an n x n row-major matrix by Gauss-Jordan with partial pivoting.
bool invert(std::vector<double>& A, int n) {
    std::vector<double> I(size_t(n) * n, 0.0);
    for (int i = 0; i < n; ++i) I[size_t(i) * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[size_t(r) * n + c]) > std::fabs(A[size_t(piv) * n + c])) piv = r;
        if (A[size_t(piv) * n + c] == 0.0) return false;
        if (piv != c)
            for (int j = 0; j < n; ++j) {
                std::swap(A[size_t(c) * n + j], A[size_t(piv) * n + j]);
                std::swap(I[size_t(c) * n + j], I[size_t(piv) * n + j]);
            }
        double d = 1.0 / A[size_t(c) * n + c];
        for (int j = 0; j < n; ++j) {
            A[size_t(c) * n + j] *= d;
            I[size_t(c) * n + j] *= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = A[size_t(r) * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[size_t(r) * n + j] -= f * A[size_t(c) * n + j];
                I[size_t(r) * n + j] -= f * I[size_t(c) * n + j];
            }
        }
    }
    A.swap(I);
    return true;
}

}  // namespace

kl_status build_direction(int p, int ne, int pt, int net, const std::vector<double>& interfaces, Direction* out) {
    if (p < 1 || ne < 1 || pt < 1 || net < 1) return fail(KL_ERR_INVALID_ARG, "degrees and element counts must be >= 1");
    if (ne + p > 4096 || net + pt > 4096) return fail(KL_ERR_INVALID_ARG, "more than 4096 functions in one direction");
    if (interfaces.size() > 64) return fail(KL_ERR_INVALID_ARG, "more than 64 patch interfaces in one direction");
    Direction& d = *out;
    d.p = p; d.ne = ne; d.pt = pt; d.net = net;
    d.itf = interfaces;
    // patch interfaces (Sec. 3.6): the trial space is C^0 there, the interpolation space C^{-1}
    Space trial, interp;
    if (!make_space_itf(p, ne, interfaces, p, &trial) || !make_space_itf(pt, net, interfaces, pt + 1, &interp))
        return fail(KL_ERR_INVALID_ARG, "a patch interface must be an interior breakpoint of both meshes");
    if (trial.n > 4096 || interp.n > 4096) return fail(KL_ERR_INVALID_ARG, "more than 4096 functions in one direction");
    d.n = trial.n;
    d.nt = interp.n;
    const int n = d.n, nt = d.nt;

    // Greville abscissae of the interpolation space; at a C^{-1} knot the function whose support
    // ends there is collocated from the left
    d.xi.assign(nt, 0.0);
    d.side.assign(nt, 0);
    for (int i = 0; i < nt; ++i) {
        double s = 0.0;
        for (int r = 1; r <= pt; ++r) s += interp.t[i + r];
        d.xi[i] = s / pt;
        if (interp.t[size_t(i + pt + 1)] == d.xi[i] && d.xi[i] > 0.0 && d.xi[i] < 1.0) d.side[i] = -1;
    }
    // Z_k (p+1 Gauss points per element) and its Cholesky factor
    std::vector<double> Z = cross_mass(trial, trial, p + 1);
    std::vector<double> Lk(size_t(n) * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double s = Z[size_t(j) * n + j];
        for (int r = 0; r < j; ++r) s -= Lk[size_t(j) * n + r] * Lk[size_t(j) * n + r];
        if (!(s > 0.0)) return fail(KL_ERR_NUMERIC, "univariate mass matrix is not positive definite");
        double ljj = std::sqrt(s);
        Lk[size_t(j) * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = Z[size_t(i) * n + j];
            for (int r = 0; r < j; ++r) t -= Lk[size_t(i) * n + r] * Lk[size_t(j) * n + r];
            Lk[size_t(i) * n + j] = t / ljj;
        }
    }
    d.L = Lk;
    // L_k^{-1} by forward substitution on the identity
    d.Linv.assign(size_t(n) * n, 0.0);
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int r = 0; r < i; ++r) s -= Lk[size_t(i) * n + r] * d.Linv[size_t(r) * n + c];
            d.Linv[size_t(i) * n + c] = s / Lk[size_t(i) * n + i];
        }
    }
    // M_k = int B~_i B_j (nt x n), exact for degree p + pt
    std::vector<double> M = cross_mass(interp, trial, (p + pt) / 2 + 1);
    // B~_k collocation (nt x nt) and its inverse
    std::vector<double> Bt(size_t(nt) * nt, 0.0), Nv(pt + 1);
    for (int i = 0; i < nt; ++i) {
        int s = d.side[i] < 0 ? find_span_left(interp.t, pt, d.xi[i]) : find_span(interp.t, pt, d.xi[i]);
        nonzero_basis(interp.t, pt, s, d.xi[i], Nv.data());
        for (int r = 0; r <= pt; ++r) Bt[size_t(i) * nt + (s - pt + r)] = Nv[r];
    }
    if (!invert(Bt, nt)) return fail(KL_ERR_NUMERIC, "collocation matrix is singular");
    // X1 = M_k L_k^{-T}  (nt x n):  X1[i][j] = sum_r M[i][r] Linv[j][r]
    std::vector<double> X1(size_t(nt) * n, 0.0);
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int r = 0; r <= j; ++r) s += M[size_t(i) * n + r] * d.Linv[size_t(j) * n + r];
            X1[size_t(i) * n + j] = s;
        }
    // C_k = B~^{-T} X1:  C[i][j] = sum_r Binv[r][i] X1[r][j]
    d.C.assign(size_t(nt) * n, 0.0);
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int r = 0; r < nt; ++r) s += Bt[size_t(r) * nt + i] * X1[size_t(r) * n + j];
            d.C[size_t(i) * n + j] = s;
        }
    return KL_OK;
}


kl_status parse_geometry(const kl_geometry* geom, NurbsMap* nm) {
    const int d = geom->dim;
    if (d < 1 || d > 3) return fail(KL_ERR_INVALID_ARG, "dim must be 1, 2 or 3");
    if (geom->kind != KL_GEOM_BOX && geom->kind != KL_GEOM_NURBS) return fail(KL_ERR_INVALID_ARG, "unsupported geometry kind");
    if (geom->kind == KL_GEOM_BOX) {
        for (int k = 0; k < d; ++k)
            if (!(geom->hi[k] > geom->lo[k]) || !std::isfinite(geom->lo[k]) || !std::isfinite(geom->hi[k]))
                return fail(KL_ERR_INVALID_ARG, "box extent must be positive");
        return KL_OK;
    }
    // NURBS map: open knot vectors on [0, 1], positive weights (host data, copied here)
    nm->dim = d;
    size_t nrec = 1;
    for (int k = 0; k < d; ++k) {
        const int p = geom->deg[k], n = geom->nctrl[k];
        if (p < 1 || p > 15 || n < p + 1 || n > 4096 || !geom->knots[k])
            return fail(KL_ERR_INVALID_ARG, "NURBS map: need 1 <= deg <= 15, nctrl >= deg + 1, knots");
        nm->deg[k] = p;
        nm->n[k] = n;
        nm->knots[k].assign(geom->knots[k], geom->knots[k] + n + p + 1);
        const std::vector<double>& t = nm->knots[k];
        for (size_t i = 0; i + 1 < t.size(); ++i)
            if (!(t[i] <= t[i + 1]) || !std::isfinite(t[i]))
                return fail(KL_ERR_INVALID_ARG, "NURBS map: knots must be finite and non-decreasing");
        for (int i = 0; i <= p; ++i)
            if (t[size_t(i)] != 0.0 || t[t.size() - 1 - size_t(i)] != 1.0)
                return fail(KL_ERR_INVALID_ARG, "NURBS map: knot vectors must be open on [0, 1]");
        nrec *= size_t(n);
    }
    if (!geom->ctrl) return fail(KL_ERR_INVALID_ARG, "NURBS map: null control points");
    nm->ctrl.assign(geom->ctrl, geom->ctrl + 4 * nrec);
    for (size_t i = 0; i < nrec; ++i) {
        for (int r = 0; r < 4; ++r)
            if (!std::isfinite(nm->ctrl[4 * i + r])) return fail(KL_ERR_INVALID_ARG, "NURBS map: non-finite control data");
        if (!(nm->ctrl[4 * i + 3] > 0.0)) return fail(KL_ERR_INVALID_ARG, "NURBS map: weights must be positive");
    }
    return KL_OK;
}

kl_status build_space(int dim, const kl_space* space, Direction* dir) {
    for (int k = 0; k < dim; ++k) {
        const int p = space->deg[k], ne = space->elems[k];
        const int pt = space->interp_deg[k] > 0 ? space->interp_deg[k] : p;
        const int net = space->interp_elems[k] > 0 ? space->interp_elems[k] : ne;
        std::vector<double> itf;
        if (space->n_interfaces[k] < 0 || (space->n_interfaces[k] > 0 && !space->interfaces[k]))
            return fail(KL_ERR_INVALID_ARG, "patch interfaces: negative count or null array");
        if (space->n_interfaces[k] > 0) itf.assign(space->interfaces[k], space->interfaces[k] + space->n_interfaces[k]);
        KL_TRY(build_direction(p, ne, pt, net, itf, &dir[k]));
    }
    return KL_OK;
}

kl_status map_greville_points(const kl_geometry* geom, const NurbsMap& nm, const Direction* dir,
                              std::vector<double>* X, std::vector<double>* J) {
    const int d = geom->dim;
    int64_t Nt = 1;
    double det = 1.0;
    for (int k = 0; k < d; ++k) {
        Nt *= dir[k].nt;
        if (geom->kind == KL_GEOM_BOX) det *= geom->hi[k] - geom->lo[k];
    }
    if (Nt > 2147483647LL) return fail(KL_ERR_INVALID_ARG, "problem too large (more than 2^31-1 points)");
    // mapped Greville points X = F(xh) in vec order (direction 1 fastest) and J = sqrt(det DF)
    X->assign(size_t(Nt) * 3, 0.0);
    J->assign(size_t(Nt), std::sqrt(det));
    // a NURBS map's basis values depend on one coordinate each: evaluate them once per
    // direction and Greville abscissa (with its side), then form every point from them
    std::vector<MapBasis1D> basis[3];
    MapBasis1D unit;
    if (geom->kind != KL_GEOM_BOX) {
        nurbs_basis_1d(nm, 3, 0.0, 0, &unit);
        for (int k = 0; k < d; ++k) {
            basis[k].resize(size_t(dir[k].nt));
            for (int i = 0; i < dir[k].nt; ++i)
                nurbs_basis_1d(nm, k, dir[k].xi[size_t(i)], dir[k].side[size_t(i)], &basis[k][size_t(i)]);
        }
    }
    // points in vec order: direction 1 fastest (nested loops, no index division)
    const int n0 = d > 0 ? dir[0].nt : 1, n1 = d > 1 ? dir[1].nt : 1, n2 = d > 2 ? dir[2].nt : 1;
    int64_t idx = 0;
    for (int i2 = 0; i2 < n2; ++i2)
        for (int i1 = 0; i1 < n1; ++i1)
            for (int i0 = 0; i0 < n0; ++i0, ++idx) {
                const int ik[3] = {i0, i1, i2};
                double* Xi = &(*X)[size_t(idx) * 3];
                if (geom->kind == KL_GEOM_BOX) {
                    for (int k = 0; k < d; ++k)
                        Xi[k] = geom->lo[k] + (geom->hi[k] - geom->lo[k]) * dir[k].xi[size_t(ik[k])];
                    continue;
                }
                const MapBasis1D* bk[3] = {&unit, &unit, &unit};
                for (int k = 0; k < d; ++k) bk[k] = &basis[k][size_t(ik[k])];
                double detDF;
                nurbs_map_from_basis(nm, bk, Xi, &detDF);
                if (!(detDF > 0.0) || !std::isfinite(detDF))
                    return fail(KL_ERR_INVALID_ARG, "NURBS map: det DF <= 0 at a Greville point (map not invertible)");
                (*J)[size_t(idx)] = std::sqrt(detDF);
            }
    return KL_OK;
}

}  // namespace kl

// host-only view of one direction's set-up (the factors kl_create uploads)
extern "C" kl_status kl_direction_factors(int deg, int elems, int interp_deg, int interp_elems, int n_interfaces,
                                          const double* interfaces, int* n, int* nt, double* greville,
                                          int* side, double* L, double* C) {
    using namespace kl;
    if (!n || !nt) return fail(KL_ERR_INVALID_ARG, "kl_direction_factors: null n or nt");
    if (n_interfaces < 0 || (n_interfaces > 0 && !interfaces))
        return fail(KL_ERR_INVALID_ARG, "patch interfaces: negative count or null array");
    const int pt = interp_deg > 0 ? interp_deg : deg;
    const int net = interp_elems > 0 ? interp_elems : elems;
    std::vector<double> itf;
    if (n_interfaces > 0) itf.assign(interfaces, interfaces + n_interfaces);
    Direction d;
    const kl_status st = build_direction(deg, elems, pt, net, itf, &d);
    if (st != KL_OK) return st;
    *n = d.n;
    *nt = d.nt;
    if (greville) std::copy(d.xi.begin(), d.xi.end(), greville);
    if (side) std::copy(d.side.begin(), d.side.end(), side);
    if (L) std::copy(d.L.begin(), d.L.end(), L);
    if (C) std::copy(d.C.begin(), d.C.end(), C);
    return KL_OK;
}

// host-only view of the standard-form prolongation of one direction (the factor kl_prolong applies)
extern "C" kl_status kl_prolongation_factor(int deg, int elems_coarse, int elems_fine, int* nc, int* nf, double* Q) {
    using namespace kl;
    if (!nc || !nf) return fail(KL_ERR_INVALID_ARG, "kl_prolongation_factor: null nc or nf");
    Direction c, f;
    KL_TRY(build_direction(deg, elems_coarse, deg, elems_coarse, {}, &c));
    KL_TRY(build_direction(deg, elems_fine, deg, elems_fine, {}, &f));
    std::vector<double> Qv;
    KL_TRY(build_prolongation(c, f, &Qv));
    *nc = c.n;
    *nf = f.n;
    if (Q) std::copy(Qv.begin(), Qv.end(), Q);
    return KL_OK;
}

// host-only view of the mapped Greville grid and J (the points kl_create uploads)
extern "C" kl_status kl_mapped_points(const kl_geometry* geom, const kl_space* space, int64_t* Ntilde, double* X,
                                      double* J) {
    using namespace kl;
    if (!geom || !space || !Ntilde) return fail(KL_ERR_INVALID_ARG, "null argument to kl_mapped_points");
    NurbsMap nm;
    KL_TRY(parse_geometry(geom, &nm));
    Direction dir[3];
    KL_TRY(build_space(geom->dim, space, dir));
    std::vector<double> Xv, Jv;
    KL_TRY(map_greville_points(geom, nm, dir, &Xv, &Jv));
    *Ntilde = int64_t(Jv.size());
    if (X) std::copy(Xv.begin(), Xv.end(), X);
    if (J) std::copy(Jv.begin(), Jv.end(), J);
    return KL_OK;
}

namespace kl {

// non-zero basis functions of direction k of the map at x, with their derivatives; side < 0
// takes the left limit (at a C^0 knot of the map)
void nurbs_basis_1d(const NurbsMap& m, int k, double x, int side, MapBasis1D* out) {
    if (k >= m.dim) {
        out->span = 0;
        out->N[0] = 1.0;
        out->dN[0] = 0.0;
        return;
    }
    out->span = side < 0 ? find_span_left(m.knots[k], m.deg[k], x) : find_span(m.knots[k], m.deg[k], x);
    nonzero_basis(m.knots[k], m.deg[k], out->span, x, out->N);
    nonzero_basis_derivative(m.knots[k], m.deg[k], out->span, x, out->dN);
}

// F(xh) and det DF(xh) of a tensor-product NURBS map (Sec. 2.4): F = P / W with
// P = sum_I N_I(xh) w_I P_I and W = sum_I N_I(xh) w_I; column j of DF is
// (dP/dxh_j W - P dW/dxh_j) / W^2.  Directions beyond dim have one control point.
void nurbs_map_from_basis(const NurbsMap& m, const MapBasis1D* const bk[3], double* X, double* detDF) {
    const double *N0 = bk[0]->N, *N1 = bk[1]->N, *N2 = bk[2]->N;
    const double *dN0 = bk[0]->dN, *dN1 = bk[1]->dN, *dN2 = bk[2]->dN;
    const int q0 = m.dim > 0 ? m.deg[0] : 0, q1 = m.dim > 1 ? m.deg[1] : 0, q2 = m.dim > 2 ? m.deg[2] : 0;
    const int o0 = m.dim > 0 ? bk[0]->span - q0 : 0, o1 = m.dim > 1 ? bk[1]->span - q1 : 0,
              o2 = m.dim > 2 ? bk[2]->span - q2 : 0;
    // homogeneous sums H = sum_I N_I(xh) w_I (P_I, 1) and their derivatives dH[j] along xh_j,
    // contracting direction 1, then 2, then 3 (the basis is a tensor product)
    double H[4] = {0, 0, 0, 0}, dH[3][4] = {{0}};
    for (int c = 0; c <= q2; ++c) {
        double B[4] = {0, 0, 0, 0}, dB0[4] = {0, 0, 0, 0}, dB1[4] = {0, 0, 0, 0};
        for (int b = 0; b <= q1; ++b) {
            double A[4] = {0, 0, 0, 0}, dA[4] = {0, 0, 0, 0};
            const double* row = &m.ctrl[4 * ((size_t(o2 + c) * m.n[1] + size_t(o1 + b)) * m.n[0] + size_t(o0))];
            for (int a = 0; a <= q0; ++a) {
                const double* cp = row + 4 * a;
                const double w = cp[3];
                const double h[4] = {w * cp[0], w * cp[1], w * cp[2], w};
                for (int r = 0; r < 4; ++r) {
                    A[r] += N0[a] * h[r];
                    dA[r] += dN0[a] * h[r];
                }
            }
            for (int r = 0; r < 4; ++r) {
                B[r] += N1[b] * A[r];
                dB0[r] += N1[b] * dA[r];
                dB1[r] += dN1[b] * A[r];
            }
        }
        for (int r = 0; r < 4; ++r) {
            H[r] += N2[c] * B[r];
            dH[0][r] += N2[c] * dB0[r];
            dH[1][r] += N2[c] * dB1[r];
            dH[2][r] += dN2[c] * B[r];
        }
    }
    const double W = H[3];
    const double P[3] = {H[0], H[1], H[2]};
    const double dW[3] = {dH[0][3], dH[1][3], dH[2][3]};
    double dP[3][3];
    for (int r = 0; r < 3; ++r)
        for (int j = 0; j < 3; ++j) dP[r][j] = dH[j][r];
    const double iW = 1.0 / W, iW2 = iW * iW;
    double D[3][3];
    for (int r = 0; r < 3; ++r) {
        X[r] = P[r] * iW;
        for (int j = 0; j < 3; ++j) D[r][j] = (dP[r][j] * W - P[r] * dW[j]) * iW2;
    }
    if (m.dim == 1) {
        *detDF = D[0][0];
    } else if (m.dim == 2) {
        *detDF = D[0][0] * D[1][1] - D[0][1] * D[1][0];
    } else {
        *detDF = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) - D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                 D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
    }
}


// Q = L_f^T P L_c^{-T} (n_f x n_c, row-major): the standard-form coefficients (Sec. 4.1) of every
// coarse trial function in the fine trial space.  The spaces have the same degree and nested
// uniform knots, so each coarse B-spline is a fine spline and P = B_f^{-1} B_c(x_f) holds its
// fine coefficients exactly (interpolation at the fine Greville points, Sec. 4.2).
kl_status build_prolongation(const Direction& c, const Direction& f, std::vector<double>* Q) {
    if (c.p != f.p) return fail(KL_ERR_INVALID_ARG, "prolongation: the spaces must have the same degree");
    if (!c.itf.empty() || !f.itf.empty())
        return fail(KL_ERR_INVALID_ARG, "prolongation: spaces with patch interfaces are not supported");
    if (f.ne % c.ne != 0) return fail(KL_ERR_INVALID_ARG, "prolongation: the fine mesh must refine the coarse one");
    const int p = c.p;
    const Space tc = make_space(p, c.ne), tf = make_space(p, f.ne);
    const int nc = tc.n, nf = tf.n;
    std::vector<double> xf(size_t(nf), 0.0);
    for (int i = 0; i < nf; ++i) {
        double s = 0.0;
        for (int r = 1; r <= p; ++r) s += tf.t[size_t(i + r)];
        xf[size_t(i)] = s / p;
    }
    std::vector<double> Bf(size_t(nf) * nf, 0.0), Bc(size_t(nf) * nc, 0.0), Nv(size_t(p) + 1);
    for (int i = 0; i < nf; ++i) {
        int s = find_span(tf.t, p, xf[size_t(i)]);
        nonzero_basis(tf.t, p, s, xf[size_t(i)], Nv.data());
        for (int r = 0; r <= p; ++r) Bf[size_t(i) * nf + (s - p + r)] = Nv[size_t(r)];
        s = find_span(tc.t, p, xf[size_t(i)]);
        nonzero_basis(tc.t, p, s, xf[size_t(i)], Nv.data());
        for (int r = 0; r <= p; ++r) Bc[size_t(i) * nc + (s - p + r)] = Nv[size_t(r)];
    }
    if (!invert(Bf, nf)) return fail(KL_ERR_NUMERIC, "prolongation: fine collocation matrix is singular");
    std::vector<double> P(size_t(nf) * nc, 0.0), T(size_t(nf) * nc, 0.0);
    for (int i = 0; i < nf; ++i)
        for (int j = 0; j < nc; ++j) {
            double s = 0.0;
            for (int r = 0; r < nf; ++r) s += Bf[size_t(i) * nf + r] * Bc[size_t(r) * nc + j];
            P[size_t(i) * nc + j] = s;
        }
    // T = P L_c^{-T}: T[i][j] = sum_r P[i][r] Linv_c[j][r]
    for (int i = 0; i < nf; ++i)
        for (int j = 0; j < nc; ++j) {
            double s = 0.0;
            for (int r = 0; r <= j; ++r) s += P[size_t(i) * nc + r] * c.Linv[size_t(j) * nc + r];
            T[size_t(i) * nc + j] = s;
        }
    // Q = L_f^T T: Q[i][j] = sum_{r >= i} L_f[r][i] T[r][j]
    Q->assign(size_t(nf) * nc, 0.0);
    for (int i = 0; i < nf; ++i)
        for (int j = 0; j < nc; ++j) {
            double s = 0.0;
            for (int r = i; r < nf; ++r) s += f.L[size_t(r) * nf + i] * T[size_t(r) * nc + j];
            (*Q)[size_t(i) * nc + j] = s;
        }
    return KL_OK;
}

}  // namespace kl
