// k_split.cu -- split-BF16 tensor-core path (placeholder until the tcgen05 kernels land).
#include "npf_internal.h"

namespace npf {

void split_term(Plan&, int, double2*) { fail(NPF_ERR_UNSUPPORTED, "split path not built yet"); }
void split_slab(Plan&, int, const int*, double2*) { fail(NPF_ERR_UNSUPPORTED, "split path not built yet"); }
void split_release(Plan&) {}

}  // namespace npf
