/*
 * CPU FP64 oracle for the matrix-free finite element action y = A(u).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline may load or run this code; the product path never does.  It shares no
 * code, header or table with the CUDA library.
 *
 * Every action routine is the plain cell-wise sum of its form: the action of
 * the bilinear (or residual) form of Eq. "generalized_bilinear_form" evaluated
 * with the quadrature sum of Eq. "poisson_action_w_quadrature", y_i = sum over
 * cells T, quadrature points q and test functions v_i of T of w_q |det J_T|
 * times the pointwise form at x_q.  Each cell is taken on its own, in order:
 * its vertex coordinates and DoFs, its affine Jacobian and determinant (affine
 * geometry is one Jacobian per cell), then per quadrature point the trial
 * values or physical gradients, the pointwise integrand, and its contribution
 * to every local test function, added straight into the global output.  The
 * forms are those of the paper's Appendix A (Mass, Laplacian, Helmholtz,
 * Elasticity, and the St. Venant-Kirchhoff hyperelastic law with its
 * linearisation), and a compressible Neo-Hookean law beside it:
 *     Psi(F) = mu/2 (tr F^T F - d) - mu ln J + lambda/2 (ln J)^2,  J = det F,
 *     P      = dPsi/dF = mu (F - F^{-T}) + lambda ln J F^{-T}.
 *
 * Conventions: tab[(k*nq + q)*nloc + j] with k = 0 the basis value and k = 1..d
 * the reference partial derivative d/dxhat_k; coords[v*dim + i];
 * cell2vertex[c*(dim+1) + m]; cell2node[c*nloc + j]; vector fields interleave
 * components, DoF = node*dim + comp.  The physical Jacobian is
 * J[i][k] = x_{v_k}[i] - x_{v_0}[i] (k = 1..d), the quadrature measure is
 * w_q |det J|.  Each routine processes cells [c0, c1) and ADDS into its outputs.
 *
 * Return codes: 0 ok, 1 a cell with det J == 0 or non-finite, 2 det F <= 0 or
 * non-finite at a quadrature point (Neo-Hookean forms only), 3 bad argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXD 3
#define ORC_MAXLOC 128

static inline const double *T(const double *tab, int nq, int nloc, int k, int q)
{
    return tab + ((long)k * nq + q) * nloc;
}

/* the cell's d+1 vertex coordinates (through the cell-to-vertex map) */
static void gather_coords(int dim, long c, const int32_t *c2v, const double *coords,
                          double X[ORC_MAXD + 1][ORC_MAXD])
{
    for (int m = 0; m <= dim; ++m)
        for (int i = 0; i < dim; ++i)
            X[m][i] = coords[(long)c2v[c * (dim + 1) + m] * dim + i];
}

/* affine geometry: J, det J, J^{-1} (one Jacobian per affine cell).  Returns 0 on a
 * singular or non-finite Jacobian. */
static int geometry(int dim, double X[ORC_MAXD + 1][ORC_MAXD], double J[ORC_MAXD][ORC_MAXD],
                    double *detJ, double Jinv[ORC_MAXD][ORC_MAXD])
{
    for (int i = 0; i < dim; ++i)
        for (int k = 0; k < dim; ++k)
            J[i][k] = X[k + 1][i] - X[0][i];
    double det;
    if (dim == 1) {
        det = J[0][0];
        if (det == 0.0 || !isfinite(det)) return 0;
        Jinv[0][0] = 1.0 / det;
    } else if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        if (det == 0.0 || !isfinite(det)) return 0;
        Jinv[0][0] = J[1][1] / det;
        Jinv[0][1] = -J[0][1] / det;
        Jinv[1][0] = -J[1][0] / det;
        Jinv[1][1] = J[0][0] / det;
    } else {
        double C[3][3]; /* cofactors */
        C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        C[0][1] = -(J[1][0] * J[2][2] - J[1][2] * J[2][0]);
        C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        C[1][0] = -(J[0][1] * J[2][2] - J[0][2] * J[2][1]);
        C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        C[1][2] = -(J[0][0] * J[2][1] - J[0][1] * J[2][0]);
        C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        C[2][1] = -(J[0][0] * J[1][2] - J[0][2] * J[1][0]);
        C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
        if (det == 0.0 || !isfinite(det)) return 0;
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k)
                Jinv[i][k] = C[k][i] / det; /* inverse = adjugate^T / det */
    }
    *detJ = det;
    return 1;
}

/* small dense helpers on d x d matrices */
static double det_small(int d, double A[ORC_MAXD][ORC_MAXD])
{
    if (d == 1) return A[0][0];
    if (d == 2) return A[0][0] * A[1][1] - A[0][1] * A[1][0];
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
         - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
         + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

static void inv_small(int d, double A[ORC_MAXD][ORC_MAXD], double det, double B[ORC_MAXD][ORC_MAXD])
{
    if (d == 1) { B[0][0] = 1.0 / det; return; }
    if (d == 2) {
        B[0][0] = A[1][1] / det;  B[0][1] = -A[0][1] / det;
        B[1][0] = -A[1][0] / det; B[1][1] = A[0][0] / det;
        return;
    }
    B[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
    B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    B[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
    B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    B[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
    B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
}

/* evaluation phase for a vector field with nc components: reference derivative
 * gh[c][k] = sum_j Phi_{k+1}[q][j] l[j][c] */
static void eval_ref_grad(int dim, int nc, int nloc, int nq, const double *tab, int q,
                          const double *l, double gh[ORC_MAXD][ORC_MAXD])
{
    for (int c = 0; c < nc; ++c)
        for (int k = 0; k < dim; ++k) {
            const double *phi = T(tab, nq, nloc, k + 1, q);
            double s = 0.0;
            for (int j = 0; j < nloc; ++j) s += phi[j] * l[j * nc + c];
            gh[c][k] = s;
        }
}

/* physical gradient G[c][i] = sum_k gh[c][k] Jinv[k][i] */
static void to_physical(int dim, int nc, double gh[ORC_MAXD][ORC_MAXD],
                        double Jinv[ORC_MAXD][ORC_MAXD], double G[ORC_MAXD][ORC_MAXD])
{
    for (int c = 0; c < nc; ++c)
        for (int i = 0; i < dim; ++i) {
            double s = 0.0;
            for (int k = 0; k < dim; ++k) s += gh[c][k] * Jinv[k][i];
            G[c][i] = s;
        }
}

/* quadrature phase for a stress-like S[c][i] tested against grad v:
 * S : grad v = sum_{c,k} dv_c/dxhat_k (sum_i S[c][i] Jinv[k][i]); the bracket is
 * e[c][k], and out[j][c] += sum_k Phi_{k+1}[q][j] e[c][k] * (w_q |det J|). */
static void quad_stress(int dim, int nloc, int nq, const double *tab, int q, double scale,
                        double S[ORC_MAXD][ORC_MAXD], double Jinv[ORC_MAXD][ORC_MAXD],
                        double *out)
{
    double e[ORC_MAXD][ORC_MAXD];
    for (int c = 0; c < dim; ++c)
        for (int k = 0; k < dim; ++k) {
            double s = 0.0;
            for (int i = 0; i < dim; ++i) s += S[c][i] * Jinv[k][i];
            e[c][k] = s * scale;
        }
    for (int k = 0; k < dim; ++k) {
        const double *psi = T(tab, nq, nloc, k + 1, q);
        for (int j = 0; j < nloc; ++j)
            for (int c = 0; c < dim; ++c) out[j * dim + c] += psi[j] * e[c][k];
    }
}

static void gather_dofs(int nc, int nloc, long c, const int32_t *c2n, const double *u, double *l)
{
    for (int j = 0; j < nloc; ++j)
        for (int m = 0; m < nc; ++m) l[j * nc + m] = u[(long)c2n[c * nloc + j] * nc + m];
}

static void scatter_dofs(int nc, int nloc, long c, const int32_t *c2n, const double *out, double *y)
{
    for (int j = 0; j < nloc; ++j)
        for (int m = 0; m < nc; ++m) y[(long)c2n[c * nloc + j] * nc + m] += out[j * nc + m];
}

static int check_args(int dim, int nloc)
{
    return dim >= 1 && dim <= ORC_MAXD && nloc >= 1 && nloc <= ORC_MAXLOC;
}

/* ---------------------------------------------------------------- Mass
 * a(u, v) = int u v dx (Appendix A, Mass).  e = w_q |det J| u(x_q). */
int orc_mass(int dim, int nloc, int nq, const double *wts, const double *tab,
             const int32_t *c2v, const double *coords, const int32_t *c2n,
             const double *u, double *y, long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[ORC_MAXLOC], out[ORC_MAXLOC];
    for (long c = c0; c < c1; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(1, nloc, c, c2n, u, l);
        if (!geometry(dim, X, J, &detJ, Jinv)) return 1;
        for (int j = 0; j < nloc; ++j) out[j] = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double *phi = T(tab, nq, nloc, 0, q);
            double uq = 0.0;
            for (int j = 0; j < nloc; ++j) uq += phi[j] * l[j];
            double e = uq * wts[q] * fabs(detJ);
            for (int j = 0; j < nloc; ++j) out[j] += phi[j] * e;
        }
        scatter_dofs(1, nloc, c, c2n, out, y);
    }
    return 0;
}

/* ---------------------------------------------------------------- Elasticity
 * a(u, v) = int sigma(u) : eps(v) dx, sigma = lambda tr(eps) I + 2 mu eps
 * (Appendix A, Elasticity); sigma is symmetric so sigma : eps(v) = sigma : grad v. */
int orc_elasticity(int dim, int nloc, int nq, const double *wts, const double *tab,
                   const int32_t *c2v, const double *coords, const int32_t *c2n,
                   double lambda, double mu, const double *u, double *y, long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[ORC_MAXLOC * ORC_MAXD], out[ORC_MAXLOC * ORC_MAXD];
    double gh[ORC_MAXD][ORC_MAXD], G[ORC_MAXD][ORC_MAXD], eps[ORC_MAXD][ORC_MAXD], sig[ORC_MAXD][ORC_MAXD];
    for (long c = c0; c < c1; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(dim, nloc, c, c2n, u, l);
        if (!geometry(dim, X, J, &detJ, Jinv)) return 1;
        for (int j = 0; j < nloc * dim; ++j) out[j] = 0.0;
        for (int q = 0; q < nq; ++q) {
            eval_ref_grad(dim, dim, nloc, nq, tab, q, l, gh);
            to_physical(dim, dim, gh, Jinv, G);
            double tr = 0.0;
            for (int i = 0; i < dim; ++i) tr += G[i][i];
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) eps[a][b] = 0.5 * (G[a][b] + G[b][a]);
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b)
                    sig[a][b] = 2.0 * mu * eps[a][b] + (a == b ? lambda * tr : 0.0);
            quad_stress(dim, nloc, nq, tab, q, wts[q] * fabs(detJ), sig, Jinv, out);
        }
        scatter_dofs(dim, nloc, c, c2n, out, y);
    }
    return 0;
}

/* Neo-Hookean pointwise quantities at one quadrature point from the physical
 * displacement gradient G: F = I + G, Jd = det F, Finv = F^{-1}. */
static int nh_kinematics(int dim, double G[ORC_MAXD][ORC_MAXD], double F[ORC_MAXD][ORC_MAXD],
                         double *Jd, double Finv[ORC_MAXD][ORC_MAXD])
{
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) F[a][b] = (a == b ? 1.0 : 0.0) + G[a][b];
    double jd = det_small(dim, F);
    if (!(jd > 0.0) || !isfinite(jd)) return 0;
    inv_small(dim, F, jd, Finv);
    *Jd = jd;
    return 1;
}

/* ---------------------------------------------------------------- NH residual
 * r(u; v) = int P(F) : grad v dx with P = mu (F - F^{-T}) + lambda ln J F^{-T},
 * per-cell (P0) mu and lambda; the body force is zero. */
int orc_nh_residual(int dim, int nloc, int nq, const double *wts, const double *tab,
                    const int32_t *c2v, const double *coords, const int32_t *c2n,
                    const double *mu_cell, const double *lam_cell,
                    const double *u, double *y, long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[ORC_MAXLOC * ORC_MAXD], out[ORC_MAXLOC * ORC_MAXD];
    double gh[ORC_MAXD][ORC_MAXD], G[ORC_MAXD][ORC_MAXD], F[ORC_MAXD][ORC_MAXD],
        Finv[ORC_MAXD][ORC_MAXD], P[ORC_MAXD][ORC_MAXD];
    for (long c = c0; c < c1; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(dim, nloc, c, c2n, u, l);
        const double mu = mu_cell[c], lam = lam_cell[c];
        if (!geometry(dim, X, J, &detJ, Jinv)) return 1;
        for (int j = 0; j < nloc * dim; ++j) out[j] = 0.0;
        for (int q = 0; q < nq; ++q) {
            eval_ref_grad(dim, dim, nloc, nq, tab, q, l, gh);
            to_physical(dim, dim, gh, Jinv, G);
            double Jd;
            if (!nh_kinematics(dim, G, F, &Jd, Finv)) return 2;
            const double lnJ = log(Jd);
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) /* F^{-T}[a][b] = Finv[b][a] */
                    P[a][b] = mu * (F[a][b] - Finv[b][a]) + lam * lnJ * Finv[b][a];
            quad_stress(dim, nloc, nq, tab, q, wts[q] * fabs(detJ), P, Jinv, out);
        }
        scatter_dofs(dim, nloc, c, c2n, out, y);
    }
    return 0;
}

/* ---------------------------------------------------------------- NH Jacobian action
 * a(du; v) = d/de r(u + e du; v) at e = 0 (the appendix's linearisation):
 * dP[H] = mu H + (mu - lambda ln J) F^{-T} H^T F^{-T} + lambda tr(F^{-1} H) F^{-T},
 * H = grad du.  Two trial fields are gathered: the linearisation point u and du. */
int orc_nh_jacobian(int dim, int nloc, int nq, const double *wts, const double *tab,
                    const int32_t *c2v, const double *coords, const int32_t *c2n,
                    const double *mu_cell, const double *lam_cell,
                    const double *u, const double *du, double *y, long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[ORC_MAXLOC * ORC_MAXD], dl[ORC_MAXLOC * ORC_MAXD], out[ORC_MAXLOC * ORC_MAXD];
    double gh[ORC_MAXD][ORC_MAXD], G[ORC_MAXD][ORC_MAXD], F[ORC_MAXD][ORC_MAXD],
        Finv[ORC_MAXD][ORC_MAXD], H[ORC_MAXD][ORC_MAXD], dP[ORC_MAXD][ORC_MAXD];
    for (long c = c0; c < c1; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(dim, nloc, c, c2n, u, l);
        gather_dofs(dim, nloc, c, c2n, du, dl);
        const double mu = mu_cell[c], lam = lam_cell[c];
        if (!geometry(dim, X, J, &detJ, Jinv)) return 1;
        for (int j = 0; j < nloc * dim; ++j) out[j] = 0.0;
        for (int q = 0; q < nq; ++q) {
            eval_ref_grad(dim, dim, nloc, nq, tab, q, l, gh);
            to_physical(dim, dim, gh, Jinv, G);
            eval_ref_grad(dim, dim, nloc, nq, tab, q, dl, gh);
            to_physical(dim, dim, gh, Jinv, H);
            double Jd;
            if (!nh_kinematics(dim, G, F, &Jd, Finv)) return 2;
            const double lnJ = log(Jd);
            double trFinvH = 0.0;
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) trFinvH += Finv[a][b] * H[b][a];
            /* M = F^{-T} H^T F^{-T};  M[a][b] = sum_{m,n} Finv[m][a] H[n][m] Finv[b][n] */
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) {
                    double m = 0.0;
                    for (int i = 0; i < dim; ++i)
                        for (int k = 0; k < dim; ++k) m += Finv[i][a] * H[k][i] * Finv[b][k];
                    dP[a][b] = mu * H[a][b] + (mu - lam * lnJ) * m + lam * trFinvH * Finv[b][a];
                }
            quad_stress(dim, nloc, nq, tab, q, wts[q] * fabs(detJ), dP, Jinv, out);
        }
        scatter_dofs(dim, nloc, c, c2n, out, y);
    }
    return 0;
}

/* ---------------------------------------------------------------- NH energy
 * Pi(u) = sum_c sum_q w_q |det J| Psi(F), written per cell into energy[c]. */
int orc_nh_energy(int dim, int nloc, int nq, const double *wts, const double *tab,
                  const int32_t *c2v, const double *coords, const int32_t *c2n,
                  const double *mu_cell, const double *lam_cell,
                  const double *u, double *energy, long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[ORC_MAXLOC * ORC_MAXD];
    double gh[ORC_MAXD][ORC_MAXD], G[ORC_MAXD][ORC_MAXD], F[ORC_MAXD][ORC_MAXD], Finv[ORC_MAXD][ORC_MAXD];
    for (long c = c0; c < c1; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(dim, nloc, c, c2n, u, l);
        const double mu = mu_cell[c], lam = lam_cell[c];
        if (!geometry(dim, X, J, &detJ, Jinv)) return 1;
        double e = 0.0;
        for (int q = 0; q < nq; ++q) {
            eval_ref_grad(dim, dim, nloc, nq, tab, q, l, gh);
            to_physical(dim, dim, gh, Jinv, G);
            double Jd;
            if (!nh_kinematics(dim, G, F, &Jd, Finv)) return 2;
            const double lnJ = log(Jd);
            double trC = 0.0;
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) trC += F[a][b] * F[a][b];
            double psi = 0.5 * mu * (trC - dim) - mu * lnJ + 0.5 * lam * lnJ * lnJ;
            e += wts[q] * fabs(detJ) * psi;
        }
        energy[c] += e;
    }
    return 0;
}

/* ---------------------------------------------------------------- NH adjoint
 * For the residual r(u; mu, lambda): JTw = J(u)^T w, and per cell
 * dmu[c] = w . dr/dmu_c = int_c (F - F^{-T}) : grad w,
 * dlam[c] = w . dr/dlambda_c = int_c ln J F^{-T} : grad w.
 * J^T w is formed literally: the element tangent K_e[(j,a),(m,b)] =
 * sum_q w_q |det J| sum_{i,k} dphi_j/dx_i A[a][i][b][k] dphi_m/dx_k with the
 * fourth-order tangent A = dP/dF, A[a][i][b][k] = mu d_ab d_ik
 * + (mu - lambda ln J) Finv[i][b] Finv[k][a] + lambda Finv[i][a] Finv[k][b],
 * then (J^T w)_e = K_e^T w_e is scattered. */
int orc_nh_adjoint(int dim, int nloc, int nq, const double *wts, const double *tab,
                   const int32_t *c2v, const double *coords, const int32_t *c2n,
                   const double *mu_cell, const double *lam_cell,
                   const double *u, const double *w, double *jtw, double *dmu, double *dlam,
                   long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    enum { NMAX = ORC_MAXLOC * ORC_MAXD };
    const int nd = nloc * dim;
    double *K = (double *)malloc(sizeof(double) * (size_t)nd * nd); /* element tangent, per call */
    if (!K) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[NMAX], wl[NMAX], out[NMAX];
    double gh[ORC_MAXD][ORC_MAXD], G[ORC_MAXD][ORC_MAXD], F[ORC_MAXD][ORC_MAXD],
        Finv[ORC_MAXD][ORC_MAXD], W[ORC_MAXD][ORC_MAXD];
    double dphi[ORC_MAXLOC][ORC_MAXD];
    int rc = 0;
    for (long c = c0; c < c1 && rc == 0; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(dim, nloc, c, c2n, u, l);
        gather_dofs(dim, nloc, c, c2n, w, wl);
        const double mu = mu_cell[c], lam = lam_cell[c];
        if (!geometry(dim, X, J, &detJ, Jinv)) { rc = 1; break; }
        for (int r = 0; r < nd * nd; ++r) K[r] = 0.0;
        double smu = 0.0, slam = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double meas = wts[q] * fabs(detJ);
            eval_ref_grad(dim, dim, nloc, nq, tab, q, l, gh);
            to_physical(dim, dim, gh, Jinv, G);
            eval_ref_grad(dim, dim, nloc, nq, tab, q, wl, gh);
            to_physical(dim, dim, gh, Jinv, W);
            double Jd;
            if (!nh_kinematics(dim, G, F, &Jd, Finv)) { rc = 2; break; }
            const double lnJ = log(Jd);
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) {
                    smu += meas * (F[a][b] - Finv[b][a]) * W[a][b];
                    slam += meas * lnJ * Finv[b][a] * W[a][b];
                }
            /* physical basis gradients */
            for (int j = 0; j < nloc; ++j)
                for (int i = 0; i < dim; ++i) {
                    double s = 0.0;
                    for (int k = 0; k < dim; ++k) s += T(tab, nq, nloc, k + 1, q)[j] * Jinv[k][i];
                    dphi[j][i] = s;
                }
            for (int j = 0; j < nloc; ++j)
                for (int a = 0; a < dim; ++a)
                    for (int m = 0; m < nloc; ++m)
                        for (int b = 0; b < dim; ++b) {
                            double s = 0.0;
                            for (int i = 0; i < dim; ++i)
                                for (int k = 0; k < dim; ++k) {
                                    double A = (a == b && i == k ? mu : 0.0)
                                             + (mu - lam * lnJ) * Finv[i][b] * Finv[k][a]
                                             + lam * Finv[i][a] * Finv[k][b];
                                    s += dphi[j][i] * A * dphi[m][k];
                                }
                            K[(size_t)(j * dim + a) * nd + m * dim + b] += meas * s;
                        }
        }
        if (rc) break;
        for (int s = 0; s < nd; ++s) {
            double acc = 0.0;
            for (int r = 0; r < nd; ++r) acc += K[(size_t)r * nd + s] * wl[r];
            out[s] = acc;
        }
        scatter_dofs(dim, nloc, c, c2n, out, jtw);
        dmu[c] += smu;
        dlam[c] += slam;
    }
    free(K);
    return rc;
}

/* ---------------------------------------------------------------- Laplacian
 * a(u, v) = int grad u . grad v dx (Appendix A, Laplacian), scalar u, v.
 * Per point: the physical gradient g = J^{-T} (reference gradient); the test
 * side needs grad v . g = sum_k dv/dxhat_k (sum_i g_i Jinv[k][i]). */
static void scalar_grad(int dim, int nloc, int nq, const double *tab, int q, const double *l,
                        double Jinv[ORC_MAXD][ORC_MAXD], double g[ORC_MAXD])
{
    double gh[ORC_MAXD][ORC_MAXD], G[ORC_MAXD][ORC_MAXD];
    eval_ref_grad(dim, 1, nloc, nq, tab, q, l, gh);
    to_physical(dim, 1, gh, Jinv, G);
    for (int i = 0; i < dim; ++i) g[i] = G[0][i];
}

static void quad_scalar_grad(int dim, int nloc, int nq, const double *tab, int q, double scale,
                             const double g[ORC_MAXD], double Jinv[ORC_MAXD][ORC_MAXD], double *out)
{
    for (int k = 0; k < dim; ++k) {
        double e = 0.0;
        for (int i = 0; i < dim; ++i) e += g[i] * Jinv[k][i];
        const double *psi = T(tab, nq, nloc, k + 1, q);
        for (int j = 0; j < nloc; ++j) out[j] += psi[j] * e * scale;
    }
}

int orc_laplace(int dim, int nloc, int nq, const double *wts, const double *tab,
                const int32_t *c2v, const double *coords, const int32_t *c2n,
                const double *u, double *y, long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[ORC_MAXLOC], out[ORC_MAXLOC], g[ORC_MAXD];
    for (long c = c0; c < c1; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(1, nloc, c, c2n, u, l);
        if (!geometry(dim, X, J, &detJ, Jinv)) return 1;
        for (int j = 0; j < nloc; ++j) out[j] = 0.0;
        for (int q = 0; q < nq; ++q) {
            scalar_grad(dim, nloc, nq, tab, q, l, Jinv, g);
            quad_scalar_grad(dim, nloc, nq, tab, q, wts[q] * fabs(detJ), g, Jinv, out);
        }
        scatter_dofs(1, nloc, c, c2n, out, y);
    }
    return 0;
}

/* ---------------------------------------------------------------- Helmholtz
 * a(u, v) = int (grad u . grad v + u v) dx (Appendix A, Helmholtz). */
int orc_helmholtz(int dim, int nloc, int nq, const double *wts, const double *tab,
                  const int32_t *c2v, const double *coords, const int32_t *c2n,
                  const double *u, double *y, long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[ORC_MAXLOC], out[ORC_MAXLOC], g[ORC_MAXD];
    for (long c = c0; c < c1; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(1, nloc, c, c2n, u, l);
        if (!geometry(dim, X, J, &detJ, Jinv)) return 1;
        for (int j = 0; j < nloc; ++j) out[j] = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double scale = wts[q] * fabs(detJ);
            const double *phi = T(tab, nq, nloc, 0, q);
            double uq = 0.0;
            for (int j = 0; j < nloc; ++j) uq += phi[j] * l[j];
            for (int j = 0; j < nloc; ++j) out[j] += phi[j] * uq * scale;
            scalar_grad(dim, nloc, nq, tab, q, l, Jinv, g);
            quad_scalar_grad(dim, nloc, nq, tab, q, scale, g, Jinv, out);
        }
        scatter_dofs(1, nloc, c, c2n, out, y);
    }
    return 0;
}

/* St. Venant-Kirchhoff law (Appendix A, Hyperelasticity): from the physical
 * displacement gradient G, F = I + G, C = F^T F, E = (C - I)/2,
 * S = dPsi/dE = lambda tr(E) I + 2 mu E for Psi = lambda/2 (tr E)^2 + mu tr(E^2),
 * P = F S.  Returns Psi. */
static double svk_stress(int dim, double G[ORC_MAXD][ORC_MAXD], double mu, double lam,
                         double F[ORC_MAXD][ORC_MAXD], double S[ORC_MAXD][ORC_MAXD],
                         double P[ORC_MAXD][ORC_MAXD])
{
    double E[ORC_MAXD][ORC_MAXD];
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) F[a][b] = (a == b ? 1.0 : 0.0) + G[a][b];
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
            double cab = 0.0;   /* C[a][b] = sum_m F[m][a] F[m][b] */
            for (int m = 0; m < dim; ++m) cab += F[m][a] * F[m][b];
            E[a][b] = 0.5 * (cab - (a == b ? 1.0 : 0.0));
        }
    double trE = 0.0, trE2 = 0.0;
    for (int a = 0; a < dim; ++a) trE += E[a][a];
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) trE2 += E[a][b] * E[b][a];
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) S[a][b] = 2.0 * mu * E[a][b] + (a == b ? lam * trE : 0.0);
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
            double p = 0.0;
            for (int m = 0; m < dim; ++m) p += F[a][m] * S[m][b];
            P[a][b] = p;
        }
    return 0.5 * lam * trE * trE + mu * trE2;
}

/* ---------------------------------------------------------------- SVK residual
 * r(u; v) = int P(F) : grad v dx, P = F S (body force zero), per-cell mu, lambda. */
int orc_svk_residual(int dim, int nloc, int nq, const double *wts, const double *tab,
                     const int32_t *c2v, const double *coords, const int32_t *c2n,
                     const double *mu_cell, const double *lam_cell,
                     const double *u, double *y, long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[ORC_MAXLOC * ORC_MAXD], out[ORC_MAXLOC * ORC_MAXD];
    double gh[ORC_MAXD][ORC_MAXD], G[ORC_MAXD][ORC_MAXD], F[ORC_MAXD][ORC_MAXD], S[ORC_MAXD][ORC_MAXD],
        P[ORC_MAXD][ORC_MAXD];
    for (long c = c0; c < c1; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(dim, nloc, c, c2n, u, l);
        const double mu = mu_cell[c], lam = lam_cell[c];
        if (!geometry(dim, X, J, &detJ, Jinv)) return 1;
        for (int j = 0; j < nloc * dim; ++j) out[j] = 0.0;
        for (int q = 0; q < nq; ++q) {
            eval_ref_grad(dim, dim, nloc, nq, tab, q, l, gh);
            to_physical(dim, dim, gh, Jinv, G);
            svk_stress(dim, G, mu, lam, F, S, P);
            quad_stress(dim, nloc, nq, tab, q, wts[q] * fabs(detJ), P, Jinv, out);
        }
        scatter_dofs(dim, nloc, c, c2n, out, y);
    }
    return 0;
}

/* ---------------------------------------------------------------- SVK Jacobian action
 * a(du; v) = d/de r(u + e du; v) at e = 0:  dP = H S + F dS, H = grad du,
 * dE = (H^T F + F^T H)/2, dS = lambda tr(dE) I + 2 mu dE. */
int orc_svk_jacobian(int dim, int nloc, int nq, const double *wts, const double *tab,
                     const int32_t *c2v, const double *coords, const int32_t *c2n,
                     const double *mu_cell, const double *lam_cell,
                     const double *u, const double *du, double *y, long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[ORC_MAXLOC * ORC_MAXD], dl[ORC_MAXLOC * ORC_MAXD], out[ORC_MAXLOC * ORC_MAXD];
    double gh[ORC_MAXD][ORC_MAXD], G[ORC_MAXD][ORC_MAXD], F[ORC_MAXD][ORC_MAXD], S[ORC_MAXD][ORC_MAXD],
        P[ORC_MAXD][ORC_MAXD], H[ORC_MAXD][ORC_MAXD], dE[ORC_MAXD][ORC_MAXD], dS[ORC_MAXD][ORC_MAXD],
        dP[ORC_MAXD][ORC_MAXD];
    for (long c = c0; c < c1; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(dim, nloc, c, c2n, u, l);
        gather_dofs(dim, nloc, c, c2n, du, dl);
        const double mu = mu_cell[c], lam = lam_cell[c];
        if (!geometry(dim, X, J, &detJ, Jinv)) return 1;
        for (int j = 0; j < nloc * dim; ++j) out[j] = 0.0;
        for (int q = 0; q < nq; ++q) {
            eval_ref_grad(dim, dim, nloc, nq, tab, q, l, gh);
            to_physical(dim, dim, gh, Jinv, G);
            eval_ref_grad(dim, dim, nloc, nq, tab, q, dl, gh);
            to_physical(dim, dim, gh, Jinv, H);
            svk_stress(dim, G, mu, lam, F, S, P);
            double trdE = 0.0;
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) {
                    double s = 0.0;   /* (H^T F + F^T H)[a][b] / 2 */
                    for (int m = 0; m < dim; ++m) s += H[m][a] * F[m][b] + F[m][a] * H[m][b];
                    dE[a][b] = 0.5 * s;
                }
            for (int a = 0; a < dim; ++a) trdE += dE[a][a];
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) dS[a][b] = 2.0 * mu * dE[a][b] + (a == b ? lam * trdE : 0.0);
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) {
                    double s = 0.0;
                    for (int m = 0; m < dim; ++m) s += H[a][m] * S[m][b] + F[a][m] * dS[m][b];
                    dP[a][b] = s;
                }
            quad_stress(dim, nloc, nq, tab, q, wts[q] * fabs(detJ), dP, Jinv, out);
        }
        scatter_dofs(dim, nloc, c, c2n, out, y);
    }
    return 0;
}

/* ---------------------------------------------------------------- SVK energy
 * Pi(u) = sum_c sum_q w_q |det J| Psi(E), per cell into energy[c]. */
int orc_svk_energy(int dim, int nloc, int nq, const double *wts, const double *tab,
                   const int32_t *c2v, const double *coords, const int32_t *c2n,
                   const double *mu_cell, const double *lam_cell,
                   const double *u, double *energy, long c0, long c1)
{
    if (!check_args(dim, nloc)) return 3;
    double X[ORC_MAXD + 1][ORC_MAXD], J[ORC_MAXD][ORC_MAXD], Jinv[ORC_MAXD][ORC_MAXD], detJ;
    double l[ORC_MAXLOC * ORC_MAXD];
    double gh[ORC_MAXD][ORC_MAXD], G[ORC_MAXD][ORC_MAXD], F[ORC_MAXD][ORC_MAXD], S[ORC_MAXD][ORC_MAXD],
        P[ORC_MAXD][ORC_MAXD];
    for (long c = c0; c < c1; ++c) {
        gather_coords(dim, c, c2v, coords, X);
        gather_dofs(dim, nloc, c, c2n, u, l);
        const double mu = mu_cell[c], lam = lam_cell[c];
        if (!geometry(dim, X, J, &detJ, Jinv)) return 1;
        double e = 0.0;
        for (int q = 0; q < nq; ++q) {
            eval_ref_grad(dim, dim, nloc, nq, tab, q, l, gh);
            to_physical(dim, dim, gh, Jinv, G);
            e += wts[q] * fabs(detJ) * svk_stress(dim, G, mu, lam, F, S, P);
        }
        energy[c] += e;
    }
    return 0;
}
