// inst_n13.cu -- kernels for N = 2^13; transform shapes: 2^12 words/CTA x 2^4 words/thread, 2^13 words/CTA x 2^4 words/thread, 2^12 words/CTA x 2^3 words/thread, 2^11 words/CTA x 2^4 words/thread.
#include "inst.cuh"

#define HE_SHAPES_13 {{12, 4}, {13, 4}, {12, 3}, {11, 4}}
namespace he {
HE_DEGREE(13, 12, 4, HE_SHAPES_13, HE_SHAPE_FN(13, 12, 4) HE_SHAPE_FN(13, 13, 4) HE_SHAPE_FN(13, 12, 3) HE_SHAPE_FN(13, 11, 4))
}  // namespace he

HE_DEFINE_DEGREE_OPS(13)
