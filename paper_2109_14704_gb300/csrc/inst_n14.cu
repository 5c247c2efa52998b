// inst_n14.cu -- kernels for N = 2^14 (words per CTA: 2^12, 2^13, 2^11).
#include "inst.cuh"

namespace he {
HE_DEGREE(14, 12, HE_SHAPE_FN(14, 12) HE_SHAPE_FN(14, 13) HE_SHAPE_FN(14, 11))
}  // namespace he

HE_DEFINE_DEGREE_OPS(14)
