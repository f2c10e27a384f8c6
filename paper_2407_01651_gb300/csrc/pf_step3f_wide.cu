// pf_step3f_wide.cu -- the periodic variants of the 3-D two-phase step kernel
// with 64-bit site indices and plane offsets, for grids whose state planes
// hold more than 2^32 elements; compiled apart so that the sets build in
// parallel.
#include "pf_step3f.cuh"

namespace pf {
namespace d3f {

PF3F_LAUNCH_SET(, false, unsigned long long)

}  // namespace d3f
}  // namespace pf
