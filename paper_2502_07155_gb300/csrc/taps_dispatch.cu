// Selection of the short-sum kernel instantiation for a plan's m.
#include "plan_internal.h"

namespace nfftbl {

template <typename T, int D>
nfftbl_status run_taps_d(nfftbl_plan_s* p, const TapArgs<T>& args, int kind, size_t smem) {
    switch (p->m) {
#define NFFTBL_CASE(M) \
    case M: return launch_tap_kernel<T, D, 2 * M>(p, args, kind, smem);
        NFFTBL_FIXED_M_LIST(NFFTBL_CASE)
#undef NFFTBL_CASE
        default:
            if (p->m < 2 || p->m > 12) return fail(p, NFFTBL_EUNSUPPORTED, "m outside 2..12");
            return launch_tap_kernel<T, D, 0>(p, args, kind, smem);
    }
}

template nfftbl_status run_taps_d<float, 1>(nfftbl_plan_s*, const TapArgs<float>&, int, size_t);
template nfftbl_status run_taps_d<float, 2>(nfftbl_plan_s*, const TapArgs<float>&, int, size_t);
template nfftbl_status run_taps_d<float, 3>(nfftbl_plan_s*, const TapArgs<float>&, int, size_t);
template nfftbl_status run_taps_d<double, 1>(nfftbl_plan_s*, const TapArgs<double>&, int, size_t);
template nfftbl_status run_taps_d<double, 2>(nfftbl_plan_s*, const TapArgs<double>&, int, size_t);
template nfftbl_status run_taps_d<double, 3>(nfftbl_plan_s*, const TapArgs<double>&, int, size_t);

}  // namespace nfftbl
