// pf_step3f_bc.cu -- the boundary-aware variants of the 3-D two-phase step
// kernel (k_step3f with BC = true: non-periodic sides), compiled apart from
// the periodic ones so that the sets build in parallel.
#include "pf_step3f.cuh"

namespace pf {
namespace d3f {

PF3F_LAUNCH_SET(, true, unsigned long long)

}  // namespace d3f
}  // namespace pf
