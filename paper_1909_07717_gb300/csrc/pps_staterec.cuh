// pps_staterec.cuh -- a state's derived constants and scaled opponents
// (derive_state and load_opps, the same values), prepared once a call by a
// thread a state for the kernels whose items come from many states in turn
// (the proposal's refinement, the batched plans), which then load them
// instead of deriving them item by item.
#pragma once

#include "pps_search.cuh"

namespace pps {

template <int JMAX>
struct __align__(16) StateRec {
    StateK sk;
    OppRegs<JMAX> o;
};

template <int JMAX>
__device__ __forceinline__ void make_state_rec(const pps_state& st,
                                               const pps_params& prm, int kmax,
                                               StateRec<JMAX>& r) {
    r.sk = derive_state(st, prm, JMAX, kmax);
    load_opps<JMAX>(st, r.sk, r.o);
}

}  // namespace pps
