// Cells-per-CTA variants of the Laplacian, Helmholtz and St. Venant-Kirchhoff
// forms for every dimension and contraction type; degree and rule are runtime
// values.
#include "fe_coop.cuh"

namespace fe {

int register_variants_coop_forms(Variant *out, int cap)
{
    const Variant v[] = {
        make_coop_variant<OP_LAPLACE, 2, double>(),        make_coop_variant<OP_LAPLACE, 3, double>(),
        make_coop_variant<OP_HELMHOLTZ, 2, double>(),      make_coop_variant<OP_HELMHOLTZ, 3, double>(),
        make_coop_variant<OP_SVK_RESIDUAL, 2, double>(),   make_coop_variant<OP_SVK_RESIDUAL, 3, double>(),
        make_coop_variant<OP_SVK_JACOBIAN, 2, double>(),   make_coop_variant<OP_SVK_JACOBIAN, 3, double>(),
        make_coop_variant<OP_LAPLACE, 2, float>(),         make_coop_variant<OP_LAPLACE, 3, float>(),
        make_coop_variant<OP_HELMHOLTZ, 2, float>(),       make_coop_variant<OP_HELMHOLTZ, 3, float>(),
        make_coop_variant<OP_SVK_RESIDUAL, 2, float>(),    make_coop_variant<OP_SVK_RESIDUAL, 3, float>(),
        make_coop_variant<OP_SVK_JACOBIAN, 2, float>(),    make_coop_variant<OP_SVK_JACOBIAN, 3, float>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
