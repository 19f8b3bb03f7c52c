// Tensor-core variants with split binary16 operands (hi + lo pairs, three
// products per term; FE_PREC_FP16X2) for every tensor-core form, 2D and 3D.
#include "fe_tc.cuh"

namespace fe {

int register_variants_tc2(Variant *out, int cap)
{
    const Variant v[] = {
        make_tc_variant<OP_MASS, 2, __half, 2>(),          make_tc_variant<OP_MASS, 3, __half, 2>(),
        make_tc_variant<OP_ELASTICITY, 2, __half, 2>(),    make_tc_variant<OP_ELASTICITY, 3, __half, 2>(),
        make_tc_variant<OP_LAPLACE, 2, __half, 2>(),       make_tc_variant<OP_LAPLACE, 3, __half, 2>(),
        make_tc_variant<OP_HELMHOLTZ, 2, __half, 2>(),     make_tc_variant<OP_HELMHOLTZ, 3, __half, 2>(),
        make_tc_variant<OP_NH_JACOBIAN, 2, __half, 2>(),   make_tc_variant<OP_NH_JACOBIAN, 3, __half, 2>(),
        make_tc_variant<OP_SVK_JACOBIAN, 2, __half, 2>(),  make_tc_variant<OP_SVK_JACOBIAN, 3, __half, 2>(),
    };
    int n = 0;
    for (const Variant &x : v)
        if (n < cap) out[n++] = x;
    return n;
}

}  // namespace fe
