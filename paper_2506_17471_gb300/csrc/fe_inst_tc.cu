// Tensor-core variants (16-bit contractions): mass, Laplacian, Helmholtz, linear
// elasticity and the Neo-Hookean and St. Venant-Kirchhoff Jacobian actions in 2D
// and 3D, BF16 and FP16; degree and rule are runtime values.
#include "fe_tc.cuh"

namespace fe {

int register_variants_tc(Variant *out, int cap)
{
    const Variant v[] = {
        make_tc_variant<OP_MASS, 2, __nv_bfloat16>(),       make_tc_variant<OP_MASS, 3, __nv_bfloat16>(),
        make_tc_variant<OP_ELASTICITY, 2, __nv_bfloat16>(), make_tc_variant<OP_ELASTICITY, 3, __nv_bfloat16>(),
        make_tc_variant<OP_MASS, 2, __half>(),              make_tc_variant<OP_MASS, 3, __half>(),
        make_tc_variant<OP_ELASTICITY, 2, __half>(),        make_tc_variant<OP_ELASTICITY, 3, __half>(),
        make_tc_variant<OP_NH_JACOBIAN, 2, __nv_bfloat16>(), make_tc_variant<OP_NH_JACOBIAN, 3, __nv_bfloat16>(),
        make_tc_variant<OP_NH_JACOBIAN, 2, __half>(),       make_tc_variant<OP_NH_JACOBIAN, 3, __half>(),
        make_tc_variant<OP_LAPLACE, 2, __nv_bfloat16>(),    make_tc_variant<OP_LAPLACE, 3, __nv_bfloat16>(),
        make_tc_variant<OP_LAPLACE, 2, __half>(),           make_tc_variant<OP_LAPLACE, 3, __half>(),
        make_tc_variant<OP_HELMHOLTZ, 2, __nv_bfloat16>(),  make_tc_variant<OP_HELMHOLTZ, 3, __nv_bfloat16>(),
        make_tc_variant<OP_HELMHOLTZ, 2, __half>(),         make_tc_variant<OP_HELMHOLTZ, 3, __half>(),
        make_tc_variant<OP_SVK_JACOBIAN, 2, __nv_bfloat16>(), make_tc_variant<OP_SVK_JACOBIAN, 3, __nv_bfloat16>(),
        make_tc_variant<OP_SVK_JACOBIAN, 2, __half>(),      make_tc_variant<OP_SVK_JACOBIAN, 3, __half>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
