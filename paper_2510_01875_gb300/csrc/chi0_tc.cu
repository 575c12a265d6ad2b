// Split-precision chi0 on the tcgen05 tensor cores (see the kernel below).
#include "lrt_internal.h"

namespace lrt {

lrt_status launch_chi0_split(const lrt_ctx* c, QData& q, cudaStream_t s) {
  (void)c; (void)q; (void)s;
  set_error("split-precision chi0 not built yet");
  return LRT_EUNSUPPORTED;
}

}  // namespace lrt
