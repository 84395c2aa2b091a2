// Fused tensor-core path (placeholder until the kernel lands).
#include "pmf_tc.cuh"

namespace pmf {

int tc_supported(const pmf_config*, std::string* why) {
  *why = "tensor-core path not built";
  return PMF_ERR_UNSUPPORTED;
}
int tc_build_tables(const pmf_config*, TcTables*, std::string* why) {
  *why = "tensor-core path not built";
  return PMF_ERR_UNSUPPORTED;
}
void tc_free_tables(TcTables*) {}
int tc_prior(const Dims&, DevState*, const double*, float*, double*, cudaStream_t) { return 0; }
int tc_step(const Dims&, const pmf_config&, const TcTables*, const MeasParams*, const TimeConsts*,
            DevState*, float*, float*, cudaStream_t) {
  return 0;
}

}  // namespace pmf
