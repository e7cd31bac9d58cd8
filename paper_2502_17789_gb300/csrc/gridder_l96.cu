// Gridder kernels for 96 x 96 subgrids (see gridder_kernels.cuh).
#include "gridder_kernels.cuh"

namespace idg {

template int gridder_launch<96>(const GridArgs&, int, int, void*);
template int gridder_configure<96>(int, int*);
template int gridder_launch_multi<96>(const GridArgs*, const int2*, int, bool, int, void*);

}  // namespace idg
