// Instantiation of the pair kernels for one and two species with the
// standard weight exponents s_f = 2 and s_c = 2 fixed at compile time (a
// separate translation unit, so that the two sets compile in parallel).
#include "k_pair_impl.cuh"

namespace tdpd {

void launch_pair_std(const PairArgs &a, cudaStream_t st, int part)
{
    if (a.nl) {
        if (a.ns == 1) launch_ns<1, true, true>(a, st, part);
        else launch_ns<2, true, true>(a, st, part);
    } else {
        if (a.ns == 1) launch_ns<1, false, true>(a, st, part);
        else launch_ns<2, false, true>(a, st, part);
    }
}

}  // namespace tdpd
