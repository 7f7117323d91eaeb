// Compiled shapes with two kernel terms, one integral state per slot, 1-2 slots.
#include "gpss_kernels.cuh"
namespace gpss {
OpTable ops_2_1_0() { return make_ops<Shape<2, 1, 0>>(); }
OpTable ops_2_2_0() { return make_ops<Shape<2, 2, 0>>(); }
}  // namespace gpss
