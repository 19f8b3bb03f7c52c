// Thread-per-cell variants that take weight-folded tables (rows of point q scaled
// by sqrt(w_q)): the FP64 linear forms (mass, elasticity, Laplacian, Helmholtz).  Registered ahead of the plain
// variants, so plans take them; the no-allocation entry point, which stages the
// caller's unfolded tables, keeps the plain ones.
#include "fe_kernels.cuh"

namespace fe {

int register_variants_fold(Variant *out, int cap)
{
    const Variant v[] = {
        make_tpc_variant<OP_MASS, 2, 1, double, true>(),
        make_tpc_variant<OP_MASS, 2, 2, double, true>(),
        make_tpc_variant<OP_MASS, 2, 3, double, true>(),
        make_tpc_variant<OP_MASS, 2, 4, double, true>(),
        make_tpc_variant<OP_MASS, 2, 5, double, true>(),
        make_tpc_variant<OP_MASS, 2, 6, double, true>(),
        make_tpc_variant<OP_MASS, 3, 1, double, true>(),
        make_tpc_variant<OP_MASS, 3, 2, double, true>(),
        make_tpc_variant<OP_MASS, 3, 3, double, true>(),
        make_tpc_variant<OP_MASS, 3, 4, double, true>(),
        make_tpc_variant<OP_ELASTICITY, 2, 1, double, true>(),
        make_tpc_variant<OP_ELASTICITY, 2, 2, double, true>(),
        make_tpc_variant<OP_ELASTICITY, 2, 3, double, true>(),
        make_tpc_variant<OP_ELASTICITY, 2, 4, double, true>(),
        make_tpc_variant<OP_ELASTICITY, 3, 1, double, true>(),
        make_tpc_variant<OP_ELASTICITY, 3, 2, double, true>(),
        make_tpc_variant<OP_LAPLACE, 2, 1, double, true>(),
        make_tpc_variant<OP_LAPLACE, 2, 2, double, true>(),
        make_tpc_variant<OP_LAPLACE, 2, 3, double, true>(),
        make_tpc_variant<OP_LAPLACE, 2, 4, double, true>(),
        make_tpc_variant<OP_LAPLACE, 3, 1, double, true>(),
        make_tpc_variant<OP_LAPLACE, 3, 2, double, true>(),
        make_tpc_variant<OP_HELMHOLTZ, 2, 1, double, true>(),
        make_tpc_variant<OP_HELMHOLTZ, 2, 2, double, true>(),
        make_tpc_variant<OP_HELMHOLTZ, 2, 3, double, true>(),
        make_tpc_variant<OP_HELMHOLTZ, 2, 4, double, true>(),
        make_tpc_variant<OP_HELMHOLTZ, 3, 1, double, true>(),
        make_tpc_variant<OP_HELMHOLTZ, 3, 2, double, true>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
