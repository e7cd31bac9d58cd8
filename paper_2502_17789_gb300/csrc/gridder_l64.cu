// Gridder kernels for 64 x 64 subgrids (see gridder_kernels.cuh).
#include "gridder_kernels.cuh"

namespace idg {

template int gridder_launch<64>(const GridArgs&, int, int, void*);
template int gridder_configure<64>(int, int*);
template int gridder_launch_multi<64>(const GridArgs*, const int2*, int, bool, int, void*);

}  // namespace idg
