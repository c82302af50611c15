// Entry points of the extensions, completed in their own translation units.
#include "nx_internal.cuh"

extern "C" nx_status nx_run_multi(nx_graph**, uint32_t, nx_program, float, uint32_t,
                                  nx_run_stats*) {
  return nx::invalid("nx_run_multi: not available in this build");
}
