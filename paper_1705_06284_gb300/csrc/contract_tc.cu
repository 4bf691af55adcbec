// Tensor-core (tcgen05) contraction: placeholder until the kernel lands.
#include "fbs_internal.h"

namespace fbs {

void launch_contract_tc(Plan &, const float *, long long, long long) {
    throw Failure{FBS_ERR_STATE, "tensor-core contraction not available in this build"};
}

void free_tc_state(Plan &) {}

}  // namespace fbs
