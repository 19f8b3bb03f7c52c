// Thread-per-cell variants of the Laplacian, Helmholtz and St. Venant-Kirchhoff
// forms (FP64 and FP32 contractions) for the degrees whose per-cell state fits
// in registers; other degrees use the cells-per-CTA variants.
#include "fe_kernels.cuh"

namespace fe {

int register_variants_forms(Variant *out, int cap)
{
    const Variant v[] = {
        make_tpc_variant<OP_LAPLACE, 2, 1, double>(),       make_tpc_variant<OP_LAPLACE, 2, 2, double>(),
        make_tpc_variant<OP_LAPLACE, 2, 3, double>(),       make_tpc_variant<OP_LAPLACE, 2, 4, double>(),
        make_tpc_variant<OP_LAPLACE, 3, 1, double>(),       make_tpc_variant<OP_LAPLACE, 3, 2, double>(),
        make_tpc_variant<OP_LAPLACE, 2, 2, float>(),        make_tpc_variant<OP_LAPLACE, 2, 4, float>(),
        make_tpc_variant<OP_LAPLACE, 3, 2, float>(),
        make_tpc_variant<OP_HELMHOLTZ, 2, 1, double>(),     make_tpc_variant<OP_HELMHOLTZ, 2, 2, double>(),
        make_tpc_variant<OP_HELMHOLTZ, 2, 3, double>(),     make_tpc_variant<OP_HELMHOLTZ, 2, 4, double>(),
        make_tpc_variant<OP_HELMHOLTZ, 3, 1, double>(),     make_tpc_variant<OP_HELMHOLTZ, 3, 2, double>(),
        make_tpc_variant<OP_HELMHOLTZ, 2, 4, float>(),      make_tpc_variant<OP_HELMHOLTZ, 3, 2, float>(),
        make_tpc_variant<OP_SVK_RESIDUAL, 2, 1, double>(),  make_tpc_variant<OP_SVK_RESIDUAL, 2, 2, double>(),
        make_tpc_variant<OP_SVK_RESIDUAL, 2, 3, double>(),  make_tpc_variant<OP_SVK_RESIDUAL, 3, 1, double>(),
        make_tpc_variant<OP_SVK_RESIDUAL, 3, 2, double>(),
        make_tpc_variant<OP_SVK_JACOBIAN, 2, 1, double>(),  make_tpc_variant<OP_SVK_JACOBIAN, 2, 2, double>(),
        make_tpc_variant<OP_SVK_JACOBIAN, 2, 3, double>(),  make_tpc_variant<OP_SVK_JACOBIAN, 3, 1, double>(),
        make_tpc_variant<OP_SVK_RESIDUAL, 2, 2, float>(),   make_tpc_variant<OP_SVK_JACOBIAN, 2, 2, float>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
