// inst_n15.cu -- kernels for N = 2^15 (words per CTA: 2^12, 2^13).
#include "inst.cuh"

namespace he {
HE_DEGREE(15, 12, HE_SHAPE_FN(15, 12) HE_SHAPE_FN(15, 13))
}  // namespace he

HE_DEFINE_DEGREE_OPS(15)
