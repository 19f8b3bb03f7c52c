// Cooperative (cells-per-CTA) variants for every operation, dimension and
// contraction type; degree and rule are runtime values.
#include "fe_coop.cuh"

namespace fe {

int register_variants_coop(Variant *out, int cap)
{
    const Variant v[] = {
        make_coop_variant<OP_MASS, 2, double>(),        make_coop_variant<OP_MASS, 3, double>(),
        make_coop_variant<OP_ELASTICITY, 2, double>(),  make_coop_variant<OP_ELASTICITY, 3, double>(),
        make_coop_variant<OP_NH_RESIDUAL, 2, double>(), make_coop_variant<OP_NH_RESIDUAL, 3, double>(),
        make_coop_variant<OP_NH_JACOBIAN, 2, double>(), make_coop_variant<OP_NH_JACOBIAN, 3, double>(),
        make_coop_variant<OP_NH_ADJOINT, 2, double>(),  make_coop_variant<OP_NH_ADJOINT, 3, double>(),
        make_coop_variant<OP_MASS, 2, float>(),         make_coop_variant<OP_MASS, 3, float>(),
        make_coop_variant<OP_ELASTICITY, 2, float>(),   make_coop_variant<OP_ELASTICITY, 3, float>(),
        make_coop_variant<OP_NH_RESIDUAL, 2, float>(),  make_coop_variant<OP_NH_RESIDUAL, 3, float>(),
        make_coop_variant<OP_NH_JACOBIAN, 2, float>(),  make_coop_variant<OP_NH_JACOBIAN, 3, float>(),
        make_coop_variant<OP_NH_ADJOINT, 2, float>(),   make_coop_variant<OP_NH_ADJOINT, 3, float>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
