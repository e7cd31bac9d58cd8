// Degridder kernels for 96 x 96 subgrids (see degridder_kernels.cuh).
#include "degridder_kernels.cuh"

namespace idg {

template int launch_degridder_l<96>(const DegridArgs&, int, int, int, void*, bool);
template int configure_degridder_l<96>(int, int, int*);
template int launch_degridder_multi_l<96>(int, bool, const DegridArgs*, const int2*, int, int, void*);

}  // namespace idg
