// Tensor-core degridder kernels for 32 x 32 subgrids (see degridder_tc_kernels.cuh).
#include "degridder_tc_kernels.cuh"

namespace idg {

template int launch_degridder_tc_l<32>(const DegridArgs&, int, int, void*);
template int configure_degridder_tc_l<32>(int, int*);
template int launch_degridder_tc_multi_l<32>(const DegridArgs*, const int2*, int, int, void*);

}  // namespace idg
