// gn_adjoint.cu -- reverse mode of the unrolled iteration (gn_backward).
#include "gn_internal.cuh"

void gn_free_record(gn_graph* g) { (void)g; }

extern "C" gn_status gn_backward(gn_graph* g, const float* dL_dxT, float* dL_dw, float* dL_dx0) {
  (void)dL_dxT; (void)dL_dw; (void)dL_dx0;
  if (!g) return gn::fail(GN_ERR_ARG, "gn_backward: NULL handle");
  return gn::fail(GN_ERR_NO_RECORD, "gn_backward: no recorded forward run");
}
