// generated by build.py: instances of pass_kernel for MODE_NLL, S = 4
#include "pass_kernel.cuh"
#include "pwa_internal.h"
namespace pwa {
KernelFn pick_pass_nll_s4(int W, int kpw)
{
    (void)kpw;  // no second sweep
    if (W == 1) return pass_kernel<MODE_NLL, 4, 1, 1>;
    if (W == 2) return pass_kernel<MODE_NLL, 4, 2, 1>;
    if (W == 4) return pass_kernel<MODE_NLL, 4, 4, 1>;
    if (W == 8) return pass_kernel<MODE_NLL, 4, 8, 1>;
    return nullptr;
}
}  // namespace pwa
