// Compiled shape with two kernel terms and one integral state per term (one slot).
#include "gpss_kernels.cuh"
namespace gpss {
OpTable ops_2_1_1() { return make_ops<Shape<2, 1, 1>>(); }
}  // namespace gpss
