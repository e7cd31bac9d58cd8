// Gridder kernels for 32 x 32 subgrids (see gridder_kernels.cuh).
#include "gridder_kernels.cuh"

namespace idg {

template int gridder_launch<32>(const GridArgs&, int, int, void*);
template int gridder_configure<32>(int, int*);
template int gridder_launch_multi<32>(const GridArgs*, const int2*, int, bool, int, void*);

}  // namespace idg
