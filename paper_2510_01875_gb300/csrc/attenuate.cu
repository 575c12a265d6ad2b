// Attenuation of narrow-band fluctuations (Sec. 3).
#include "lrt_internal.h"

namespace lrt {

lrt_status run_attenuation(const lrt_ctx* c, const lrt_atten_params* p, const double* S_dev,
                           double* Sp_host, lrt_atten_report* rep, cudaStream_t s) {
  (void)c; (void)p; (void)S_dev; (void)Sp_host; (void)rep; (void)s;
  set_error("attenuation not built yet");
  return LRT_EUNSUPPORTED;
}

}  // namespace lrt
