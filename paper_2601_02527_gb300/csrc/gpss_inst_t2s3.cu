// Compiled shape with two kernel terms and three slots (augmented dimension 7).
#include "gpss_kernels.cuh"
namespace gpss {
OpTable ops_2_3_0() { return make_ops<Shape<2, 3, 0>>(); }
}  // namespace gpss
