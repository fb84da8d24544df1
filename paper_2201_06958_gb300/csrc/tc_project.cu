// tc_project.cu - placeholder until the tensor-core projection lands.
#include "tc_project.h"

namespace tdb {

bool tc_supported(int, const int64_t*, const int*, std::string& err) {
  err = "not built yet";
  return false;
}
void tc_carve(TcPlan&, Carver&, int, const int64_t*, const int*) {}
tdb_status tc_project(TcPlan&, const float*, const float*, int, const int64_t*, const int*, const void* const*, float*,
                      float* const*, double*, int, const WeightView&, double*, unsigned*, cudaStream_t,
                      std::string& err) {
  err = "not built yet";
  return TDB_ERR_UNSUPPORTED;
}

}  // namespace tdb
