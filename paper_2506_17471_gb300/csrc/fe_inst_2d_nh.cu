// Thread-per-cell variants, 2D Neo-Hookean residual, Jacobian action and adjoint.
#include "fe_kernels.cuh"

namespace fe {

int register_variants_2d_nh(Variant *out, int cap)
{
    const Variant v[] = {
        make_tpc_variant<OP_NH_RESIDUAL, 2, 1>(), make_tpc_variant<OP_NH_RESIDUAL, 2, 2>(),
        make_tpc_variant<OP_NH_RESIDUAL, 2, 3>(), make_tpc_variant<OP_NH_RESIDUAL, 2, 4>(),
        make_tpc_variant<OP_NH_JACOBIAN, 2, 1>(), make_tpc_variant<OP_NH_JACOBIAN, 2, 2>(),
        make_tpc_variant<OP_NH_JACOBIAN, 2, 3>(), make_tpc_variant<OP_NH_JACOBIAN, 2, 4>(),
        make_tpc_variant<OP_NH_ADJOINT, 2, 1>(),  make_tpc_variant<OP_NH_ADJOINT, 2, 2>(),
        make_tpc_variant<OP_NH_ADJOINT, 2, 3>(),  make_tpc_variant<OP_NH_ADJOINT, 2, 4>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
