// Thread-per-cell variants, 3D forms (FP64 and FP32 contractions).
#include "fe_kernels.cuh"

namespace fe {

int register_variants_3d(Variant *out, int cap)
{
    const Variant v[] = {
        make_tpc_variant<OP_MASS, 3, 1, double>(),
        make_tpc_variant<OP_MASS, 3, 2, double>(),
        make_tpc_variant<OP_MASS, 3, 3, double>(),
        make_tpc_variant<OP_MASS, 3, 4, double>(),
        make_tpc_variant<OP_MASS, 3, 1, float>(),
        make_tpc_variant<OP_MASS, 3, 2, float>(),
        make_tpc_variant<OP_MASS, 3, 3, float>(),
        make_tpc_variant<OP_MASS, 3, 4, float>(),
        make_tpc_variant<OP_ELASTICITY, 3, 1, double>(),
        make_tpc_variant<OP_ELASTICITY, 3, 2, double>(),
        make_tpc_variant<OP_ELASTICITY, 3, 1, float>(),
        make_tpc_variant<OP_ELASTICITY, 3, 2, float>(),
        make_tpc_variant<OP_NH_RESIDUAL, 3, 1, double>(),
        make_tpc_variant<OP_NH_RESIDUAL, 3, 2, double>(),
        make_tpc_variant<OP_NH_RESIDUAL, 3, 1, float>(),
        make_tpc_variant<OP_NH_RESIDUAL, 3, 2, float>(),
        make_tpc_variant<OP_NH_JACOBIAN, 3, 1, double>(),
        make_tpc_variant<OP_NH_JACOBIAN, 3, 2, double>(),
        make_tpc_variant<OP_NH_JACOBIAN, 3, 1, float>(),
        make_tpc_variant<OP_NH_JACOBIAN, 3, 2, float>(),
        make_tpc_variant<OP_NH_ADJOINT, 3, 1, double>(),
        make_tpc_variant<OP_NH_ADJOINT, 3, 2, double>(),
        make_tpc_variant<OP_NH_ADJOINT, 3, 1, float>(),
        make_tpc_variant<OP_NH_ADJOINT, 3, 2, float>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
