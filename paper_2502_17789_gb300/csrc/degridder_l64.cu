// Degridder kernels for 64 x 64 subgrids (see degridder_kernels.cuh).
#include "degridder_kernels.cuh"

namespace idg {

template int launch_degridder_l<64>(const DegridArgs&, int, int, int, void*, bool);
template int configure_degridder_l<64>(int, int, int*);
template int launch_degridder_multi_l<64>(int, bool, const DegridArgs*, const int2*, int, int, void*);

}  // namespace idg
