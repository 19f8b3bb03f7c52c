// Thread-per-cell variants, 2D Neo-Hookean residual, Jacobian action and adjoint
// (FP64 and FP32 contractions).
#include "fe_kernels.cuh"

namespace fe {

int register_variants_2d_nh(Variant *out, int cap)
{
    const Variant v[] = {
        make_tpc_variant<OP_NH_RESIDUAL, 2, 1, double>(),
        make_tpc_variant<OP_NH_RESIDUAL, 2, 2, double>(),
        make_tpc_variant<OP_NH_RESIDUAL, 2, 3, double>(),
        make_tpc_variant<OP_NH_RESIDUAL, 2, 4, double>(),
        make_tpc_variant<OP_NH_RESIDUAL, 2, 1, float>(),
        make_tpc_variant<OP_NH_RESIDUAL, 2, 2, float>(),
        make_tpc_variant<OP_NH_RESIDUAL, 2, 3, float>(),
        make_tpc_variant<OP_NH_RESIDUAL, 2, 4, float>(),
        make_tpc_variant<OP_NH_JACOBIAN, 2, 1, double>(),
        make_tpc_variant<OP_NH_JACOBIAN, 2, 2, double>(),
        make_tpc_variant<OP_NH_JACOBIAN, 2, 3, double>(),
        make_tpc_variant<OP_NH_JACOBIAN, 2, 4, double>(),
        make_tpc_variant<OP_NH_JACOBIAN, 2, 1, float>(),
        make_tpc_variant<OP_NH_JACOBIAN, 2, 2, float>(),
        make_tpc_variant<OP_NH_JACOBIAN, 2, 3, float>(),
        make_tpc_variant<OP_NH_JACOBIAN, 2, 4, float>(),
        make_tpc_variant<OP_NH_ADJOINT, 2, 1, double>(),
        make_tpc_variant<OP_NH_ADJOINT, 2, 2, double>(),
        make_tpc_variant<OP_NH_ADJOINT, 2, 3, double>(),
        make_tpc_variant<OP_NH_ADJOINT, 2, 4, double>(),
        make_tpc_variant<OP_NH_ADJOINT, 2, 1, float>(),
        make_tpc_variant<OP_NH_ADJOINT, 2, 2, float>(),
        make_tpc_variant<OP_NH_ADJOINT, 2, 3, float>(),
        make_tpc_variant<OP_NH_ADJOINT, 2, 4, float>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
