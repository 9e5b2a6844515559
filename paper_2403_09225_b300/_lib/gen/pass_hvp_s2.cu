// generated by build.py: instances of pass_kernel for MODE_HVP, S = 2
#include "pass_kernel.cuh"
#include "pwa_internal.h"
namespace pwa {
KernelFn pick_pass_hvp_s2(int W, int kpw)
{
    if (W == 1 && kpw == 1) return pass_kernel<MODE_HVP, 2, 1, 1>;
    if (W == 1 && kpw == 2) return pass_kernel<MODE_HVP, 2, 1, 2>;
    if (W == 1 && kpw == 3) return pass_kernel<MODE_HVP, 2, 1, 3>;
    if (W == 1 && kpw == 4) return pass_kernel<MODE_HVP, 2, 1, 4>;
    if (W == 1 && kpw == 5) return pass_kernel<MODE_HVP, 2, 1, 5>;
    if (W == 1 && kpw == 6) return pass_kernel<MODE_HVP, 2, 1, 6>;
    if (W == 1 && kpw == 7) return pass_kernel<MODE_HVP, 2, 1, 7>;
    if (W == 1 && kpw == 8) return pass_kernel<MODE_HVP, 2, 1, 8>;
    if (W == 2 && kpw == 1) return pass_kernel<MODE_HVP, 2, 2, 1>;
    if (W == 2 && kpw == 2) return pass_kernel<MODE_HVP, 2, 2, 2>;
    if (W == 2 && kpw == 3) return pass_kernel<MODE_HVP, 2, 2, 3>;
    if (W == 2 && kpw == 4) return pass_kernel<MODE_HVP, 2, 2, 4>;
    if (W == 2 && kpw == 5) return pass_kernel<MODE_HVP, 2, 2, 5>;
    if (W == 2 && kpw == 6) return pass_kernel<MODE_HVP, 2, 2, 6>;
    if (W == 2 && kpw == 7) return pass_kernel<MODE_HVP, 2, 2, 7>;
    if (W == 2 && kpw == 8) return pass_kernel<MODE_HVP, 2, 2, 8>;
    if (W == 4 && kpw == 1) return pass_kernel<MODE_HVP, 2, 4, 1>;
    if (W == 4 && kpw == 2) return pass_kernel<MODE_HVP, 2, 4, 2>;
    if (W == 4 && kpw == 3) return pass_kernel<MODE_HVP, 2, 4, 3>;
    if (W == 4 && kpw == 4) return pass_kernel<MODE_HVP, 2, 4, 4>;
    if (W == 4 && kpw == 5) return pass_kernel<MODE_HVP, 2, 4, 5>;
    if (W == 4 && kpw == 6) return pass_kernel<MODE_HVP, 2, 4, 6>;
    if (W == 4 && kpw == 7) return pass_kernel<MODE_HVP, 2, 4, 7>;
    if (W == 4 && kpw == 8) return pass_kernel<MODE_HVP, 2, 4, 8>;
    if (W == 8 && kpw == 1) return pass_kernel<MODE_HVP, 2, 8, 1>;
    if (W == 8 && kpw == 2) return pass_kernel<MODE_HVP, 2, 8, 2>;
    if (W == 8 && kpw == 3) return pass_kernel<MODE_HVP, 2, 8, 3>;
    if (W == 8 && kpw == 4) return pass_kernel<MODE_HVP, 2, 8, 4>;
    if (W == 8 && kpw == 5) return pass_kernel<MODE_HVP, 2, 8, 5>;
    if (W == 8 && kpw == 6) return pass_kernel<MODE_HVP, 2, 8, 6>;
    if (W == 8 && kpw == 7) return pass_kernel<MODE_HVP, 2, 8, 7>;
    if (W == 8 && kpw == 8) return pass_kernel<MODE_HVP, 2, 8, 8>;
    return nullptr;
}
}  // namespace pwa
