// pass_nll.cu -- instances of the fused pass for mode MODE_NLL (see pass_kernel.cuh).
#include "pwa_internal.h"

namespace pwa {

namespace {
template <int S>
KernelFn by_kpw(int kpw)
{
    (void)kpw;  // no second sweep: one instance per S
    return pass_kernel<MODE_NLL, S, 1>;
}
}  // namespace

KernelFn pick_pass_nll(int S, int kpw)
{
    switch (S) {
        case 1: return by_kpw<1>(kpw);
        case 2: return by_kpw<2>(kpw);
        case 3: return by_kpw<3>(kpw);
        case 4: return by_kpw<4>(kpw);
        default: return nullptr;
    }
}

}  // namespace pwa
