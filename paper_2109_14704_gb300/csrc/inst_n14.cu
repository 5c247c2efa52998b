// inst_n14.cu -- kernels for N = 2^14; transform shapes: 2^11 words/CTA x 2^4 words/thread (default: the
// key-switching kernels measured fastest with it), 2^12 x 2^4, 2^13 x 2^4, 2^12 x 2^3.
#include "inst.cuh"

#define HE_SHAPES_14 {{11, 4}, {12, 4}, {13, 4}, {12, 3}}
namespace he {
HE_DEGREE(14, 11, 4, HE_SHAPES_14, HE_SHAPE_FN(14, 11, 4) HE_SHAPE_FN(14, 12, 4) HE_SHAPE_FN(14, 13, 4) HE_SHAPE_FN(14, 12, 3))
}  // namespace he

HE_DEFINE_DEGREE_OPS(14)
