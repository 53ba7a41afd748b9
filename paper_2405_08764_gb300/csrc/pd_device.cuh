// Device helpers shared by the fused and the persistent macro-step kernels.
#pragma once

#include "pd_internal.h"

namespace pd {

constexpr unsigned kFull = 0xffffffffu;

template <typename real>
__device__ __forceinline__ void load_vec4(const real* __restrict__ p, real& x, real& y, real& z, real& w)
{
    if constexpr (sizeof(real) == 4) {
        float4 q = __ldg(reinterpret_cast<const float4*>(p));
        x = q.x; y = q.y; z = q.z; w = q.w;
    } else {
        double2 q0 = __ldg(reinterpret_cast<const double2*>(p));
        double2 q1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
        x = q0.x; y = q0.y; z = q1.x; w = q1.y;
    }
}

__device__ __forceinline__ int wrap_col(const InstDev& I, int i)
{
    if (!I.periodic) return i;
    return i < 0 ? i + I.nxp : (i >= I.nxp ? i - I.nxp : i);
}

}  // namespace pd
