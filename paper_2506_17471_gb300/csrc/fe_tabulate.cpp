// Host-side quadrature rules and reference tabulation (fe_tabulate).
//
// The action's quadrature phase replaces each cell integral by a weighted sum
// (Eq. "poisson_action_w_quadrature"); its evaluation and quadrature phases read
// the tabulated reference basis values/derivatives (Eq.
// "poisson_tabulated_values").  The paper does not name its rule, so the
// library uses the collapsed conical-product Gauss-Jacobi rule of a requested
// exactness degree q: n = ceil((q+1)/2) points per direction, direction k using
// the weight (1-t)^(d-k) on [0,1].
//
// Gauss-Jacobi nodes are found as the roots of the degree-n orthonormal Jacobi
// polynomial: sign changes are bracketed on a fine grid, then refined by
// safeguarded Newton steps; weights are Christoffel numbers
// 1 / sum_{k<n} p_k(x_i)^2 of the orthonormal family.
//
// The basis is the equispaced P_p Lagrange basis in barycentric product form
// phi_alpha = prod_m L_{alpha_m}(lam_m), L_a(s) = prod_{i<a} (p s - i)/(i+1),
// differentiated factor by factor.

#include <cmath>
#include <cstring>
#include <vector>

#include "fe_internal.h"

namespace fe {
bool symmetric_rule(int dim, int q, std::vector<double> &pts, std::vector<double> &wts);
}

namespace {

// Recurrence of the monic Jacobi polynomials for (1-x)^a (1+x)^b on [-1,1]:
// P_{k+1} = (x - alpha_k) P_k - beta_k P_{k-1}.
void jacobi_recurrence(int n, double a, double b, std::vector<double> &alpha,
                       std::vector<double> &beta, double &mu0)
{
    alpha.assign(n, 0.0);
    beta.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        const double s = 2.0 * k + a + b;
        if (k == 0)
            alpha[k] = (b - a) / (a + b + 2.0);
        else
            alpha[k] = (b * b - a * a) / (s * (s + 2.0));
        if (k >= 1) {
            const double num = 4.0 * k * (k + a) * (k + b) * (k + a + b);
            const double den = s * s * (s + 1.0) * (s - 1.0);
            beta[k] = num / den;
        }
    }
    mu0 = std::pow(2.0, a + b + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0) /
          std::tgamma(a + b + 2.0);
}

// Orthonormal polynomial values p_0..p_n at x (p_k = P_k / sqrt(beta_1..beta_k mu0)),
// returns p_n and its derivative, and sum_{k<n} p_k^2.
void orthonormal_eval(int n, const std::vector<double> &alpha, const std::vector<double> &beta,
                      double mu0, double x, double &pn, double &dpn, double &sumsq)
{
    double pm1 = 0.0, dpm1 = 0.0;
    double p = 1.0 / std::sqrt(mu0), dp = 0.0;
    sumsq = 0.0;
    for (int k = 0; k < n; ++k) {
        sumsq += p * p;
        const double sb_next = std::sqrt(k + 1 < n ? beta[k + 1] : 0.0);
        // for k+1 == n, use the unnormalised monic step scaled by 1 (roots unchanged)
        const double sb = k >= 1 ? std::sqrt(beta[k]) : 0.0;
        double pnext = (x - alpha[k]) * p - sb * pm1;
        double dpnext = p + (x - alpha[k]) * dp - sb * dpm1;
        if (k + 1 < n) {
            pnext /= sb_next;
            dpnext /= sb_next;
        }
        pm1 = p;
        dpm1 = dp;
        p = pnext;
        dp = dpnext;
    }
    pn = p;
    dpn = dp;
}

// n-point Gauss-Jacobi rule for (1-t)^a on [0,1].
void gauss_jacobi_01(int n, int a, std::vector<double> &t, std::vector<double> &w)
{
    std::vector<double> alpha, beta;
    double mu0;
    jacobi_recurrence(n, double(a), 0.0, alpha, beta, mu0);
    t.clear();
    w.clear();
    // Chebyshev-spaced scan grid with an odd count, so no grid point is x = 0
    // (a root of every odd-degree symmetric family).
    const int grid = 4000 * n + 1;
    const double kPi = 3.14159265358979323846;
    double xprev = -1.0, fprev, dtmp, stmp;
    orthonormal_eval(n, alpha, beta, mu0, xprev, fprev, dtmp, stmp);
    for (int g = 1; g <= grid && (int)t.size() < n; ++g) {
        const double x = -std::cos(kPi * g / grid);
        double f;
        orthonormal_eval(n, alpha, beta, mu0, x, f, dtmp, stmp);
        if (f == 0.0 || (f > 0) != (fprev > 0)) {
            double lo = xprev, hi = x, flo = fprev;
            double r = f == 0.0 ? x : 0.5 * (lo + hi);
            for (int it = 0; it < 200 && f != 0.0; ++it) {
                double fr, dfr, s;
                orthonormal_eval(n, alpha, beta, mu0, r, fr, dfr, s);
                if (fr == 0.0) break;
                if ((fr > 0) == (flo > 0)) { lo = r; flo = fr; } else { hi = r; }
                double rn = (dfr != 0.0) ? r - fr / dfr : 0.5 * (lo + hi);
                if (!(rn > lo && rn < hi)) rn = 0.5 * (lo + hi);
                if (std::fabs(rn - r) <= 1e-17 + 4e-16 * std::fabs(r)) { r = rn; break; }
                r = rn;
            }
            double fr, dfr, s;
            orthonormal_eval(n, alpha, beta, mu0, r, fr, dfr, s);
            t.push_back(0.5 * (1.0 + r));
            // Christoffel number on [-1,1], mapped to [0,1] with weight (1-t)^a
            w.push_back((1.0 / s) * std::pow(2.0, -double(a) - 1.0));
            if (f == 0.0) f = -fprev;  // the sign flips across a simple root
        }
        xprev = x;
        fprev = f;
    }
}

struct Rule {
    int nq = 0;
    std::vector<double> pts, wts;
};

bool simplex_rule(int dim, int q, Rule &r)
{
    const int n = (q + 2) / 2;  // ceil((q+1)/2)
    std::vector<std::vector<double>> T(dim), W(dim);
    for (int k = 0; k < dim; ++k) {
        gauss_jacobi_01(n, dim - 1 - k, T[k], W[k]);
        if ((int)T[k].size() != n) return false;
    }
    int nq = 1;
    for (int k = 0; k < dim; ++k) nq *= n;
    r.nq = nq;
    r.pts.assign((size_t)nq * dim, 0.0);
    r.wts.assign(nq, 0.0);
    for (int i = 0; i < nq; ++i) {
        // mixed-radix digits, direction 0 most significant (outermost)
        int rem = i, digit[3] = {0, 0, 0};
        for (int k = dim - 1; k >= 0; --k) { digit[k] = rem % n; rem /= n; }
        double scale = 1.0, wt = 1.0;
        for (int k = 0; k < dim; ++k) {
            const double tk = T[k][digit[k]];
            r.pts[(size_t)i * dim + k] = tk * scale;
            scale *= (1.0 - tk);
            wt *= W[k][digit[k]];
        }
        r.wts[i] = wt;
    }
    return true;
}

// Node multi-indices in the documented order (alpha_1 outermost).
void multi_indices(int dim, int p, std::vector<int> &out)
{
    out.clear();
    if (dim == 1) {
        for (int a = 0; a <= p; ++a) out.push_back(a);
    } else if (dim == 2) {
        for (int a = 0; a <= p; ++a)
            for (int b = 0; b <= p - a; ++b) { out.push_back(a); out.push_back(b); }
    } else {
        for (int a = 0; a <= p; ++a)
            for (int b = 0; b <= p - a; ++b)
                for (int c = 0; c <= p - a - b; ++c) {
                    out.push_back(a); out.push_back(b); out.push_back(c);
                }
    }
}

void tabulate_at(int dim, int p, const double *x, const std::vector<int> &mi, int nl,
                 double *val, double *grad /*[dim][nl]*/)
{
    double lam[4];
    lam[0] = 1.0;
    for (int k = 0; k < dim; ++k) { lam[k + 1] = x[k]; lam[0] -= x[k]; }
    // factor tables L[m][a], dL[m][a] for a = 0..p
    double L[4][16], dL[4][16];
    for (int m = 0; m <= dim; ++m) {
        L[m][0] = 1.0;
        dL[m][0] = 0.0;
        for (int a = 1; a <= p; ++a) {
            const double f = (p * lam[m] - (a - 1)) / a;
            L[m][a] = L[m][a - 1] * f;
            dL[m][a] = dL[m][a - 1] * f + L[m][a - 1] * (double(p) / a);
        }
    }
    for (int j = 0; j < nl; ++j) {
        int al[4];
        al[0] = p;
        for (int k = 0; k < dim; ++k) { al[k + 1] = mi[(size_t)j * dim + k]; al[0] -= al[k + 1]; }
        double v = 1.0;
        for (int m = 0; m <= dim; ++m) v *= L[m][al[m]];
        val[j] = v;
        // d/dlam_m of the product, then chain rule with dlam_0/dxhat_k = -1,
        // dlam_{k+1}/dxhat_k = 1
        double dm[4];
        for (int m = 0; m <= dim; ++m) {
            double prod = dL[m][al[m]];
            for (int mm = 0; mm <= dim; ++mm)
                if (mm != m) prod *= L[mm][al[mm]];
            dm[m] = prod;
        }
        for (int k = 0; k < dim; ++k) grad[(size_t)k * nl + j] = dm[k + 1] - dm[0];
    }
}

}  // namespace

extern "C" int fe_tabulate_scheme(int dim, int degree, int quad_degree, int scheme, int *nq, double *pts,
                                  double *wts, double *tab, size_t cap)
{
    if (dim < 1 || dim > 3 || degree < 1 || degree > 10 || quad_degree < 0 || quad_degree > 40 ||
        nq == nullptr || scheme < FE_QUAD_CONICAL || scheme > FE_QUAD_SYMMETRIC)
        return FE_ERR_INVALID_ARG;
    Rule r;
    bool have = false;
    if (scheme == FE_QUAD_SYMMETRIC && dim >= 2) {
        std::vector<double> p, w;
        if (fe::symmetric_rule(dim, quad_degree, p, w)) {
            r.nq = (int)w.size();
            r.pts = p;
            r.wts = w;
            have = true;
        }
    }
    if (!have && !simplex_rule(dim, quad_degree, r)) return FE_ERR_INVALID_ARG;
    *nq = r.nq;
    if (tab == nullptr) return FE_OK;
    if (pts == nullptr || wts == nullptr) return FE_ERR_INVALID_ARG;
    std::vector<int> mi;
    multi_indices(dim, degree, mi);
    const int nl = (int)mi.size() / dim;
    if (cap < (size_t)(1 + dim) * r.nq * nl) return FE_ERR_INVALID_ARG;
    std::memcpy(pts, r.pts.data(), sizeof(double) * r.pts.size());
    std::memcpy(wts, r.wts.data(), sizeof(double) * r.wts.size());
    std::vector<double> val(nl), grad((size_t)dim * nl);
    for (int q = 0; q < r.nq; ++q) {
        tabulate_at(dim, degree, &r.pts[(size_t)q * dim], mi, nl, val.data(), grad.data());
        for (int j = 0; j < nl; ++j) tab[(size_t)q * nl + j] = val[j];
        for (int k = 0; k < dim; ++k)
            for (int j = 0; j < nl; ++j)
                tab[((size_t)(k + 1) * r.nq + q) * nl + j] = grad[(size_t)k * nl + j];
    }
    return FE_OK;
}

extern "C" int fe_tabulate(int dim, int degree, int quad_degree, int *nq, double *pts, double *wts,
                           double *tab, size_t cap)
{
    return fe_tabulate_scheme(dim, degree, quad_degree, FE_QUAD_CONICAL, nq, pts, wts, tab, cap);
}
