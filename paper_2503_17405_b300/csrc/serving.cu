// Serving scheduler (continuous batching).
#include "engine_internal.h"

void serving_shutdown(fsmc_engine* e) { (void)e; }
void serving_forget(fsmc_job* j) { (void)j; }
extern "C" fsmc_status fsmc_submit(fsmc_engine* e, fsmc_job* j, fsmc_mode mode) {
  (void)e; (void)j; (void)mode;
  return fsmc_fail(FSMC_ESTATE, "serving scheduler not built");
}
extern "C" fsmc_status fsmc_poll(fsmc_job* j, int* done, double* latency_s) {
  (void)j; (void)done; (void)latency_s;
  return fsmc_fail(FSMC_ESTATE, "serving scheduler not built");
}
extern "C" fsmc_status fsmc_wait_all(fsmc_engine* e, double timeout_s) {
  (void)e; (void)timeout_s;
  return FSMC_OK;
}
