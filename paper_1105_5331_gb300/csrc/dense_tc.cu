// Dense MTTKRP on tcgen05 tensor cores (bf16x3 split products).
#include "cp_internal.cuh"

namespace cpg {

cp_status mttkrp_dense_mixed(cp_ctx*, cp_tensor*, const Layout&, const double*, int, double*) {
  set_error("mixed precision MTTKRP: not built yet");
  return CP_ERR_UNSUPPORTED;
}

void tensor_free_mixed(cp_tensor* t) { (void)t; }

}  // namespace cpg
