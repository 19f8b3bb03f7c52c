// Thread-per-cell variants, 2D mass and linear elasticity.
#include "fe_kernels.cuh"

namespace fe {

int register_variants_2d_linear(Variant *out, int cap)
{
    const Variant v[] = {
        make_tpc_variant<OP_MASS, 2, 1>(),       make_tpc_variant<OP_MASS, 2, 2>(),
        make_tpc_variant<OP_MASS, 2, 3>(),       make_tpc_variant<OP_MASS, 2, 4>(),
        make_tpc_variant<OP_MASS, 2, 5>(),       make_tpc_variant<OP_MASS, 2, 6>(),
        make_tpc_variant<OP_ELASTICITY, 2, 1>(), make_tpc_variant<OP_ELASTICITY, 2, 2>(),
        make_tpc_variant<OP_ELASTICITY, 2, 3>(), make_tpc_variant<OP_ELASTICITY, 2, 4>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
