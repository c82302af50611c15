// Entry points of the extensions, completed in their own translation units.
#include "nx_internal.cuh"

extern "C" nx_status nx_adjoint_wpr(nx_graph*, const float*, uint32_t, float*, float*, int32_t,
                                    nx_run_stats*) {
  return nx::invalid("nx_adjoint_wpr: not available in this build");
}
extern "C" nx_status nx_run_multi(nx_graph**, uint32_t, nx_program, float, uint32_t,
                                  nx_run_stats*) {
  return nx::invalid("nx_run_multi: not available in this build");
}
