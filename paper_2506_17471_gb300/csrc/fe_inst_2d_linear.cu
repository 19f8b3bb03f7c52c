// Thread-per-cell variants, 2D mass and linear elasticity (FP64 and FP32 contractions).
#include "fe_kernels.cuh"

namespace fe {

int register_variants_2d_linear(Variant *out, int cap)
{
    const Variant v[] = {
        make_tpc_variant<OP_MASS, 2, 1, double>(),
        make_tpc_variant<OP_MASS, 2, 2, double>(),
        make_tpc_variant<OP_MASS, 2, 3, double>(),
        make_tpc_variant<OP_MASS, 2, 4, double>(),
        make_tpc_variant<OP_MASS, 2, 5, double>(),
        make_tpc_variant<OP_MASS, 2, 6, double>(),
        make_tpc_variant<OP_MASS, 2, 1, float>(),
        make_tpc_variant<OP_MASS, 2, 2, float>(),
        make_tpc_variant<OP_MASS, 2, 3, float>(),
        make_tpc_variant<OP_MASS, 2, 4, float>(),
        make_tpc_variant<OP_MASS, 2, 5, float>(),
        make_tpc_variant<OP_MASS, 2, 6, float>(),
        make_tpc_variant<OP_ELASTICITY, 2, 1, double>(),
        make_tpc_variant<OP_ELASTICITY, 2, 2, double>(),
        make_tpc_variant<OP_ELASTICITY, 2, 3, double>(),
        make_tpc_variant<OP_ELASTICITY, 2, 4, double>(),
        make_tpc_variant<OP_ELASTICITY, 2, 1, float>(),
        make_tpc_variant<OP_ELASTICITY, 2, 2, float>(),
        make_tpc_variant<OP_ELASTICITY, 2, 3, float>(),
        make_tpc_variant<OP_ELASTICITY, 2, 4, float>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
