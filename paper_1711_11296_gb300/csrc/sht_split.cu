// Split-precision (BF16/FP16 tensor-core) Legendre path.
#include "sht_internal.h"

namespace sht {

struct SplitTables {};

cudaError_t split_tables_create(sht_plan_s*, cudaStream_t) {
    set_error("split-precision plans are not available in this build");
    return cudaErrorNotSupported;
}
void split_tables_destroy(sht_plan_s* p) { delete p->split; p->split = nullptr; }
cudaError_t launch_legendre_fwd_split(const sht_plan_s*, const void*, void*, cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_legendre_inv_split(const sht_plan_s*, const void*, void*, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace sht
