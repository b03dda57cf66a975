// Instantiation of the pair kernels with exponents read per replica, the
// half shell's finishing pass, and the dispatch (the kernels themselves are
// in k_pair_impl.cuh).
#include "k_pair_impl.cuh"

namespace tdpd {

void launch_pair_finish(const PairArgs &a, cudaStream_t st)
{
    const int g = (a.n + 255) / 256;
    switch (a.qr ? 0 : a.ns) {
    case 1: launch_pdl(k_pair_finish<1>, g, 256, st, a); break;
    case 2: launch_pdl(k_pair_finish<2>, g, 256, st, a); break;
    case 10: launch_pdl(k_pair_finish<10>, g, 256, st, a); break;
    default: launch_pdl(k_pair_finish<0>, g, 256, st, a); break;
    }
}

void launch_pair(const PairArgs &a, cudaStream_t st, int part)
{
    if (a.n <= 0) return;
    if (a.std_exp && !a.qr && (a.ns == 1 || a.ns == 2)) {
        launch_pair_std(a, st, part);
    } else if (a.qr) {
        // the random flux lives in the general kernel only
        if (a.nl) launch_ns<0, true, false>(a, st, part);
        else launch_ns<0, false, false>(a, st, part);
    } else if (a.nl) {
        switch (a.ns) {
        case 1: launch_ns<1, true, false>(a, st, part); break;
        case 2: launch_ns<2, true, false>(a, st, part); break;
        case 10: launch_ns<10, true, false>(a, st, part); break;     // the paper's ten-species case
        default: launch_ns<0, true, false>(a, st, part); break;
        }
    } else {
        switch (a.ns) {
        case 1: launch_ns<1, false, false>(a, st, part); break;
        case 2: launch_ns<2, false, false>(a, st, part); break;
        default: launch_ns<0, false, false>(a, st, part); break;
        }
    }
}

}  // namespace tdpd
