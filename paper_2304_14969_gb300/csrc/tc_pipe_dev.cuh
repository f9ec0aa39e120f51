// Device helpers shared by the pipelined tensor-core block kernels
// (k_tc_pipe.cu, k_tc_pipe7.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qsim_internal.h"

namespace qs {

// One 32-byte global store (sm_100 and later; p 32-byte aligned).
__device__ __forceinline__ void st_global_256(void *p, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t a4,
                                              uint32_t a5, uint32_t a6, uint32_t a7)
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a0), "r"(a1), "r"(a2),
                 "r"(a3), "r"(a4), "r"(a5), "r"(a6), "r"(a7)
                 : "memory");
}

// Amplitude index of tile t's base: t's bits spread over the non-tile
// qubits (the NT tile qubits P.tpos[] get 0).
template <int NT>
__device__ __forceinline__ uint64_t tile_base(const TcPipeArgs &P, uint64_t t)
{
    uint64_t base = t;
#pragma unroll
    for (int j = 0; j < NT; j++) {
        const int p = P.tpos[j];
        base = ((base >> p) << (p + 1)) | (base & ((1ull << p) - 1));
    }
    return base;
}

// sin and cos of 2 pi tt / 2^64 (tt: a phase in 64-bit fixed-point turns).
__device__ __forceinline__ void turns_sincos(uint64_t tt, float &s, float &c)
{
    const float f = (float)(int64_t)tt * 5.42101086242752217e-20f;   // turns in [-0.5, 0.5)
    sincospif(2.0f * f, &s, &c);
}

}  // namespace qs
