// pass_grad.cu -- instances of the fused pass for mode MODE_GRAD (see pass_kernel.cuh).
#include "pwa_internal.h"

namespace pwa {

namespace {
template <int S>
KernelFn by_kpw(int kpw)
{
    switch (kpw) {
        case 1: return pass_kernel<MODE_GRAD, S, 1>;
        case 2: return pass_kernel<MODE_GRAD, S, 2>;
        case 3: return pass_kernel<MODE_GRAD, S, 3>;
        case 4: return pass_kernel<MODE_GRAD, S, 4>;
        case 5: return pass_kernel<MODE_GRAD, S, 5>;
        case 6: return pass_kernel<MODE_GRAD, S, 6>;
        case 8: return pass_kernel<MODE_GRAD, S, 8>;
        default: return nullptr;
    }
}
}  // namespace

KernelFn pick_pass_grad(int S, int kpw)
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
