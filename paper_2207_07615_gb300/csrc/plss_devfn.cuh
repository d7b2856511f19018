// plss_devfn.cuh -- device helpers shared by the sweep kernels of the
// single- and many-right-hand-side paths.
#pragma once

#include <cuda_runtime.h>

namespace plss {

// Double-float accumulator (an unevaluated sum hi + lo of two floats, about
// 48 significant bits) built from FP32 operations only. The FP32-storage
// sweeps keep their inner products in it: on GB300 every FP64
// warp-instruction holds the SM's FP64 pipe for about twenty cycles whether
// or not all lanes are active, so per-row FP64 epilogues would bound those
// sweeps. Only the CTA total is converted to double.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

// a + x * y with the product split exactly (x*y = p + fma(x, y, -p)).
__device__ __forceinline__ DF df_add_prod(DF a, float x, float y) {
    const float p = __fmul_rn(x, y);
    return df_add(a, DF{p, fmaf(x, y, -p)});
}

// Programmatic dependent launch: the sweeps are launched so that a kernel
// may start while its predecessor drains; everything it reads was written
// by that predecessor, so it first waits for the predecessor's completion
// (griddepcontrol.wait returns at once when there is none).
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace plss
