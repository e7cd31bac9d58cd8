// Gridder kernels for 128 x 128 subgrids (see gridder_kernels.cuh).
#include "gridder_kernels.cuh"

namespace idg {

template int gridder_launch<128>(const GridArgs&, int, int, void*);
template int gridder_configure<128>(int, int*);
template int gridder_launch_multi<128>(const GridArgs*, const int2*, int, bool, int, void*);

}  // namespace idg
