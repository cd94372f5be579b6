// Tensor-core (tcgen05) DFT-GEMM form of the open-boundary solve.
#include "sc_internal.cuh"

namespace sc {

sc_status tf32_create(sc_grid* g) {
  (void)g;
  return set_error(SC_ERR_UNSUPPORTED, "SC_SOLVE_TF32X3 is not built yet");
}
void tf32_destroy(sc_grid* g) { (void)g; }
sc_status tf32_solve(sc_grid* g) {
  (void)g;
  return set_error(SC_ERR_UNSUPPORTED, "SC_SOLVE_TF32X3 is not built yet");
}

}  // namespace sc
