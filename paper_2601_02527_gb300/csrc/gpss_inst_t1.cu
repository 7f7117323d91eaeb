// Compiled shapes with one kernel term (SHO or Matern-3/2), 1-3 slots.
#include "gpss_kernels.cuh"
namespace gpss {
OpTable ops_1_1_0() { return make_ops<Shape<1, 1, 0>>(); }
OpTable ops_1_2_0() { return make_ops<Shape<1, 2, 0>>(); }
OpTable ops_1_3_0() { return make_ops<Shape<1, 3, 0>>(); }
}  // namespace gpss
