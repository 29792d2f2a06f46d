// Mixed-precision form: FP64 outer defect correction around FP32 inner V-cycles.
#include "mpfc_internal.h"

size_t mpfc_fp32_carve(mpfc_s* H, const mpfc_params* p, size_t* off, char* base, int nlev) {
  (void)H; (void)p; (void)off; (void)base; (void)nlev;
  return 0;
}
int mpfc_fp32_init(mpfc_s* H) { (void)H; return MPFC_OK; }
void mpfc_fp32_destroy(mpfc_s* H) { (void)H; }
int mpfc_fp32_enqueue_step(mpfc_s* H, int scheme, cudaStream_t cs, cudaGraphConditionalHandle hnd) {
  (void)H; (void)scheme; (void)cs; (void)hnd;
  return MPFC_ERR_INVALID;
}
int mpfc_fp32_step_stream(mpfc_s* H, int scheme) {
  (void)H; (void)scheme;
  return MPFC_ERR_INVALID;
}
