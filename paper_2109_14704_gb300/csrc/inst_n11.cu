// inst_n11.cu -- kernels for N = 2^11 (words per CTA: 2^11, 2^10).
#include "inst.cuh"

namespace he {
HE_DEGREE(11, 11, HE_SHAPE_FN(11, 11) HE_SHAPE_FN(11, 10))
}  // namespace he

HE_DEFINE_DEGREE_OPS(11)
