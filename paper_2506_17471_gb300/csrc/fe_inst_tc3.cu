// Tensor-core variants with TF32 operands (kind::tf32, FP32 accumulation;
// FE_PREC_TF32) for every tensor-core form, 2D and 3D.
#include "fe_tc.cuh"

namespace fe {

int register_variants_tc3(Variant *out, int cap)
{
    const Variant v[] = {
        make_tc_variant<OP_MASS, 2, tf32_t>(),          make_tc_variant<OP_MASS, 3, tf32_t>(),
        make_tc_variant<OP_ELASTICITY, 2, tf32_t>(),    make_tc_variant<OP_ELASTICITY, 3, tf32_t>(),
        make_tc_variant<OP_LAPLACE, 2, tf32_t>(),       make_tc_variant<OP_LAPLACE, 3, tf32_t>(),
        make_tc_variant<OP_HELMHOLTZ, 2, tf32_t>(),     make_tc_variant<OP_HELMHOLTZ, 3, tf32_t>(),
        make_tc_variant<OP_NH_JACOBIAN, 2, tf32_t>(),   make_tc_variant<OP_NH_JACOBIAN, 3, tf32_t>(),
        make_tc_variant<OP_SVK_JACOBIAN, 2, tf32_t>(),  make_tc_variant<OP_SVK_JACOBIAN, 3, tf32_t>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
