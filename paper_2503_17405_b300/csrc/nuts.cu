// NUTS as a finite state machine (filled in below the ESS / DR path).
#include "engine_internal.h"
#include "fsmc_kernels.h"

void nuts_layout(fsmc_job* j, size_t& off) { (void)j; (void)off; }
fsmc_status nuts_init_state(fsmc_job* j, cudaStream_t st) {
  (void)j; (void)st;
  return fsmc_fail(FSMC_EINVAL, "NUTS kernels are not built in this library");
}
cudaError_t nuts_fsm_round(fsmc_job* j, cudaStream_t st) { (void)j; (void)st; return cudaErrorNotSupported; }
fsmc_status nuts_run_sync(fsmc_job* j, cudaStream_t st) {
  (void)j; (void)st;
  return fsmc_fail(FSMC_EINVAL, "NUTS kernels are not built in this library");
}
