// inst_n13.cu -- kernels for N = 2^13 (words per CTA: 2^12, 2^13, 2^11).
#include "inst.cuh"

namespace he {
HE_DEGREE(13, 12, HE_SHAPE_FN(13, 12) HE_SHAPE_FN(13, 13) HE_SHAPE_FN(13, 11))
}  // namespace he

HE_DEFINE_DEGREE_OPS(13)
