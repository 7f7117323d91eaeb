// Compiled shapes without integral states: series of instantaneous
// measurements (Section 2), one or two kernel terms.
#include "gpss_kernels.cuh"
namespace gpss {
OpTable ops_1_0_0() { return make_ops<Shape<1, 0, 0>>(); }
OpTable ops_2_0_0() { return make_ops<Shape<2, 0, 0>>(); }
}  // namespace gpss
