// Product-kernel models (instantaneous measurements; plain filters).
#include "gpss_prod.cuh"
namespace gpss {
OpTable ops_prod1() { return make_prod_ops<false>(); }
OpTable ops_prod2() { return make_prod_ops<true>(); }
}  // namespace gpss
