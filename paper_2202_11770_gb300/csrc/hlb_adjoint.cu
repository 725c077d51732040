// hlb_adjoint.cu — discrete adjoint of the fused step (in progress).
#include "hlb_internal.h"

extern "C" int hlb_adjoint_workspace_bytes(const hlb_solver* h, int64_t nsteps, int64_t n_probe, size_t* bytes) {
  (void)h; (void)nsteps; (void)n_probe; (void)bytes;
  return hlb_fail(HLB_ERR_STATE, "adjoint not available yet");
}
extern "C" int hlb_adjoint_run(hlb_solver* h, int64_t nsteps, const hlb_objective* obj, void* ws, size_t ws_bytes,
                               double* J, double* dtau, double* damp) {
  (void)h; (void)nsteps; (void)obj; (void)ws; (void)ws_bytes; (void)J; (void)dtau; (void)damp;
  return hlb_fail(HLB_ERR_STATE, "adjoint not available yet");
}
