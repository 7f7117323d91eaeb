// Cross-chunk combination in FP64 for the shapes with two kernel terms and
// one integral state per slot (1-2 slots), without integral states, and the
// state of dimension 6 without integral states of the product model with a
// plain term.
#include "gpss_kernels.cuh"
namespace gpss {
CombineOps comb64_2_0_0() { return make_combine<Shape<2, 0, 0>, double>(); }
CombineOps comb64_3_0_0() { return make_combine<Shape<3, 0, 0>, double>(); }
CombineOps comb64_2_1_0() { return make_combine<Shape<2, 1, 0>, double>(); }
CombineOps comb64_2_2_0() { return make_combine<Shape<2, 2, 0>, double>(); }
}  // namespace gpss
