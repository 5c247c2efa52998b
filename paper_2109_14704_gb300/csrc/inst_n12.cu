// inst_n12.cu -- kernels for N = 2^12 (words per CTA: 2^12, 2^11, 2^10).
#include "inst.cuh"

namespace he {
HE_DEGREE(12, 12, HE_SHAPE_FN(12, 12) HE_SHAPE_FN(12, 11) HE_SHAPE_FN(12, 10))
}  // namespace he

HE_DEFINE_DEGREE_OPS(12)
