// Tensor-core gridder kernels for 64 x 64 subgrids (see gridder_tc_kernels.cuh).
#include "gridder_tc_kernels.cuh"

namespace idg {

template int configure_gridder_tc_l<64>(int*);
template int launch_gridder_tc_l<64>(const GridArgs&, int, int, void*);
template int launch_gridder_tc_multi_l<64>(const GridArgs*, const int2*, int, void*);
template int launch_stage_tc_l<64>(const StageArgs&, const SegmentDesc*, int, void*);

}  // namespace idg
