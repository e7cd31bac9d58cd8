// Tensor-core degridder kernels for 96 x 96 subgrids (see degridder_tc_kernels.cuh).
#include "degridder_tc_kernels.cuh"

namespace idg {

template int launch_degridder_tc_l<96>(const DegridArgs&, int, int, void*);
template int configure_degridder_tc_l<96>(int, int*);
template int launch_degridder_tc_multi_l<96>(const DegridArgs*, const int2*, int, int, void*);

}  // namespace idg
