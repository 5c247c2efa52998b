// inst_n10.cu -- kernels for N = 2^10 (words per CTA: 2^10).
#include "inst.cuh"

namespace he {
HE_DEGREE(10, 10, HE_SHAPE_FN(10, 10))
}  // namespace he

HE_DEFINE_DEGREE_OPS(10)
