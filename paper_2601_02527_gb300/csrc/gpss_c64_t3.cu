// Cross-chunk combination in FP64 for the two-term shapes of augmented
// dimension 6 and 7 (one integral state per term; three slots).
#include "gpss_kernels.cuh"
namespace gpss {
CombineOps comb64_2_1_1() { return make_combine<Shape<2, 1, 1>, double>(); }
CombineOps comb64_2_3_0() { return make_combine<Shape<2, 3, 0>, double>(); }
}  // namespace gpss
