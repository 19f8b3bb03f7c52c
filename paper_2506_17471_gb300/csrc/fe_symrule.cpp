// Fully symmetric quadrature rules on the triangle and the tetrahedron.
//
// A fully symmetric rule is invariant under every permutation of the
// barycentric coordinates: its points come in orbits (the centroid; points
// with two or three distinct barycentric values), all points of an orbit
// sharing one weight.  Fewer points than the conical-product rule reach the same
// exactness (the paper's kernels use such rules: its Q column of Table
// "action_param_space" lists 12 points for degree 6 and 16 for degree 8 on
// triangles, and 23 for the degree-6 elasticity P4 tetrahedron, where the
// fully symmetric rule here has 24).  Here each rule is derived at run time:
// given an orbit structure and a rough starting point, Gauss-Newton
// (central-difference Jacobian, normal equations) drives the residual of the
// moment equations
//     sum_i w_i xhat_i^alpha = alpha! / (|alpha| + d)!     for all |alpha| <= q
// to rounding level (each equation relative to its right-hand side); the result
// is accepted only with positive weights, points strictly inside and relative
// residual below 1e-13.  Points are returned sorted
// lexicographically by (xhat_1, xhat_2, xhat_3).
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

namespace fe {
namespace {

enum Orbit { S3, S21, S111, S4, S31, S22, S211 };

struct RuleSpec {
    int dim, degree;
    std::vector<Orbit> orbits;
    std::vector<double> x0;   // per orbit: parameters, then the orbit's weight
};

int nparams(Orbit o) { return (o == S3 || o == S4) ? 0 : ((o == S111 || o == S211) ? 2 : 1); }

// Rough starting points (4 significant digits); the solve supplies the rest.
const std::vector<RuleSpec> &specs()
{
    static const std::vector<RuleSpec> s = {
        {2, 2, {S21}, {0.1667, 0.1667}},
        {2, 4, {S21, S21}, {0.4459, 0.03723, 0.09158, 0.01833}},
        {2, 6, {S21, S21, S111}, {0.2493, 0.01946, 0.06309, 0.008474, 0.05315, 0.3104, 0.006904}},
        {2, 8, {S3, S21, S21, S21, S111},
         {0.07216, 0.4593, 0.01585, 0.1706, 0.01720, 0.05055, 0.005410, 0.008395, 0.2631, 0.002269}},
        {3, 2, {S31}, {0.1382, 0.04167}},
        {3, 5, {S31, S31, S22}, {0.3109, 0.01878, 0.09274, 0.01225, 0.04550, 0.007091}},
        // degree 6, 24 points: three (a,a,a,1-3a) orbits and one (a,a,b,1-2a-b) orbit
        // (the orbit structure of Keast's positive degree-6 rule)
        {3, 6, {S31, S31, S31, S211},
         {0.2146, 0.006654, 0.04067, 0.001680, 0.3223, 0.009226, 0.06366, 0.2697, 0.008036}},
    };
    return s;
}

template <typename T>
void expand(int dim, const std::vector<Orbit> &orbits, const std::vector<T> &x, std::vector<T> &pts,
            std::vector<T> &wts)
{
    pts.clear();
    wts.clear();
    size_t i = 0;
    const T one = 1, half = T(1) / 2, third = T(1) / 3, quarter = T(1) / 4;
    auto add = [&](std::array<T, 4> lam, int nl, T w) {
        // all distinct permutations of lam[0..nl)
        std::sort(lam.begin(), lam.begin() + nl);
        do {
            for (int k = 1; k < nl; ++k) pts.push_back(lam[k]);   // xhat_k = lambda_k
            wts.push_back(w);
        } while (std::next_permutation(lam.begin(), lam.begin() + nl));
    };
    for (Orbit o : orbits) {
        const T *p = x.data() + i;
        const int np = nparams(o);
        const T w = p[np];
        i += np + 1;
        switch (o) {
        case S3: add({third, third, third, T(0)}, 3, w); break;
        case S21: add({p[0], p[0], one - 2 * p[0], T(0)}, 3, w); break;
        case S111: add({p[0], p[1], one - p[0] - p[1], T(0)}, 3, w); break;
        case S4: add({quarter, quarter, quarter, quarter}, 4, w); break;
        case S31: add({p[0], p[0], p[0], one - 3 * p[0]}, 4, w); break;
        case S22: add({p[0], p[0], half - p[0], half - p[0]}, 4, w); break;
        case S211: add({p[0], p[0], p[1], one - 2 * p[0] - p[1]}, 4, w); break;
        }
    }
    (void)dim;
}

template <typename T>
T factorial(int n)
{
    T f = 1;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

template <typename T>
T ipow(T x, int e)
{
    T r = 1;
    for (int k = 0; k < e; ++k) r *= x;
    return r;
}

template <typename T>
void residual(int dim, int q, const std::vector<Orbit> &orbits, const std::vector<T> &x, std::vector<T> &r)
{
    std::vector<T> pts, wts;
    expand(dim, orbits, x, pts, wts);
    r.clear();
    const int nq = (int)wts.size();
    for (int a = 0; a <= q; ++a)
        for (int b = 0; b + a <= q; ++b) {
            const int cmax = (dim == 3) ? q - a - b : 0;
            for (int c = 0; c <= cmax; ++c) {
                T s = 0;
                for (int i = 0; i < nq; ++i) {
                    const T *X = &pts[(size_t)i * dim];
                    T v = ipow(X[0], a) * ipow(X[1], b);
                    if (dim == 3) v *= ipow(X[2], c);
                    s += wts[i] * v;
                }
                // relative residual: high-degree moments are small, an absolute
                // tolerance would leave the orbit parameters loose
                const T exact = factorial<T>(a) * factorial<T>(b) * factorial<T>(c) / factorial<T>(a + b + c + dim);
                r.push_back(s / exact - T(1));
            }
        }
}

// Gauss-Newton in precision T from x (central-difference Jacobian, normal
// equations by Gaussian elimination with partial pivoting); keeps the best
// iterate and returns its largest relative moment residual.
template <typename T>
T gauss_newton(const RuleSpec &spec, std::vector<T> &x, int max_it, T h_rel)
{
    const int n = (int)x.size();
    std::vector<T> r, rp, rm;
    T best = 1e300L;
    std::vector<T> xbest = x;
    for (int it = 0; it < max_it; ++it) {
        residual<T>(spec.dim, spec.degree, spec.orbits, x, r);
        T rmax = 0;
        for (T v : r) rmax = std::max(rmax, v < 0 ? -v : v);
        if (rmax < best) {
            best = rmax;
            xbest = x;
        } else if (it > 20) {
            break;   // at rounding level: further steps only wander
        }
        const int m = (int)r.size();
        std::vector<T> J((size_t)m * n);
        for (int j = 0; j < n; ++j) {
            const T ax = x[j] < 0 ? -x[j] : x[j];
            const T h = h_rel * (ax > 1 ? ax : T(1));
            std::vector<T> xp = x, xm = x;
            xp[j] += h;
            xm[j] -= h;
            residual<T>(spec.dim, spec.degree, spec.orbits, xp, rp);
            residual<T>(spec.dim, spec.degree, spec.orbits, xm, rm);
            for (int i = 0; i < m; ++i) J[(size_t)i * n + j] = (rp[i] - rm[i]) / (2 * h);
        }
        std::vector<T> A((size_t)n * (n + 1), T(0));
        for (int a = 0; a < n; ++a) {
            for (int b = 0; b < n; ++b) {
                T sum = 0;
                for (int i = 0; i < m; ++i) sum += J[(size_t)i * n + a] * J[(size_t)i * n + b];
                A[(size_t)a * (n + 1) + b] = sum;
            }
            T g = 0;
            for (int i = 0; i < m; ++i) g += J[(size_t)i * n + a] * r[i];
            A[(size_t)a * (n + 1) + n] = -g;
        }
        for (int c = 0; c < n; ++c) {
            int piv = c;
            for (int k = c + 1; k < n; ++k) {
                const T u = A[(size_t)k * (n + 1) + c], v = A[(size_t)piv * (n + 1) + c];
                if ((u < 0 ? -u : u) > (v < 0 ? -v : v)) piv = k;
            }
            if (A[(size_t)piv * (n + 1) + c] == T(0)) return T(1);
            if (piv != c)
                for (int k = 0; k <= n; ++k) std::swap(A[(size_t)c * (n + 1) + k], A[(size_t)piv * (n + 1) + k]);
            for (int k = c + 1; k < n; ++k) {
                const T f = A[(size_t)k * (n + 1) + c] / A[(size_t)c * (n + 1) + c];
                for (int l = c; l <= n; ++l) A[(size_t)k * (n + 1) + l] -= f * A[(size_t)c * (n + 1) + l];
            }
        }
        std::vector<T> dx(n);
        for (int c = n - 1; c >= 0; --c) {
            T sum = A[(size_t)c * (n + 1) + n];
            for (int k = c + 1; k < n; ++k) sum -= A[(size_t)c * (n + 1) + k] * dx[k];
            dx[c] = sum / A[(size_t)c * (n + 1) + c];
        }
        for (int j = 0; j < n; ++j) x[j] += dx[j];
    }
    x = xbest;
    return best;
}

// Solve in double into the basin, polish in extended precision (long double),
// round once: each rule comes out correctly rounded to double.
bool solve(const RuleSpec &spec, std::vector<double> &x)
{
    x = spec.x0;
    gauss_newton<double>(spec, x, 200, 1e-7);
    std::vector<long double> xl(x.begin(), x.end());
    const long double res = gauss_newton<long double>(spec, xl, 60, 1e-9L);
    if (!(res < 1e-13L)) return false;
    for (size_t i = 0; i < x.size(); ++i) x[i] = (double)xl[i];
    std::vector<double> pts, wts;
    expand(spec.dim, spec.orbits, x, pts, wts);
    for (double w : wts)
        if (!(w > 0)) return false;
    for (size_t i = 0; i < wts.size(); ++i) {
        double sum = 0;
        for (int k = 0; k < spec.dim; ++k) {
            const double v = pts[i * spec.dim + k];
            if (!(v > 0)) return false;
            sum += v;
        }
        if (!(sum < 1)) return false;
    }
    return true;
}

}  // namespace

// The fully symmetric rule of the smallest tabulated degree >= q for dim
// (2 or 3): points [nq][dim] sorted lexicographically, weights [nq].  Returns
// false if none is tabulated (the caller then uses the conical-product rule).
bool symmetric_rule(int dim, int q, std::vector<double> &pts, std::vector<double> &wts)
{
    const RuleSpec *best = nullptr;
    for (const RuleSpec &s : specs())
        if (s.dim == dim && s.degree >= q && (!best || s.degree < best->degree)) best = &s;
    if (!best) return false;
    std::vector<double> x;
    if (!solve(*best, x)) return false;
    std::vector<double> p, w;
    expand(dim, best->orbits, x, p, w);
    const size_t nq = w.size();
    std::vector<size_t> order(nq);
    for (size_t i = 0; i < nq; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        for (int k = 0; k < dim; ++k) {
            const double u = p[a * dim + k], v = p[b * dim + k];
            if (u != v) return u < v;
        }
        return false;
    });
    pts.resize(nq * dim);
    wts.resize(nq);
    for (size_t i = 0; i < nq; ++i) {
        for (int k = 0; k < dim; ++k) pts[i * dim + k] = p[order[i] * dim + k];
        wts[i] = w[order[i]];
    }
    return true;
}

}  // namespace fe
