// Cross-chunk combination in FP64 (element combination, chunk
// log-likelihoods and boundary adjoints in double; Section 3.2.5) for the
// shapes with one kernel term, instantaneous or with 1-3 slots.
#include "gpss_kernels.cuh"
namespace gpss {
CombineOps comb64_1_0_0() { return make_combine<Shape<1, 0, 0>, double>(); }
CombineOps comb64_1_1_0() { return make_combine<Shape<1, 1, 0>, double>(); }
CombineOps comb64_1_2_0() { return make_combine<Shape<1, 2, 0>, double>(); }
CombineOps comb64_1_3_0() { return make_combine<Shape<1, 3, 0>, double>(); }
}  // namespace gpss
