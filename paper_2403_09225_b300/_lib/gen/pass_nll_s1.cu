// generated by build.py: instances of pass_kernel for MODE_NLL, S = 1
#include "pass_kernel.cuh"
#include "pwa_internal.h"
namespace pwa {
KernelFn pick_pass_nll_s1(int W, int kpw)
{
    (void)kpw;  // no second sweep
    if (W == 1) return pass_kernel<MODE_NLL, 1, 1, 1>;
    if (W == 2) return pass_kernel<MODE_NLL, 1, 2, 1>;
    if (W == 4) return pass_kernel<MODE_NLL, 1, 4, 1>;
    if (W == 8) return pass_kernel<MODE_NLL, 1, 8, 1>;
    return nullptr;
}
}  // namespace pwa
