// Device helpers of the 16-bit split operands of the tensor-core stages (one definition for the
// single-problem dense stages and the batched ones).
//   BF16 : hi = bf16(x), lo = bf16(x - hi); no scaling.
//   FP16 : each row is first scaled by a power of two s that puts its largest magnitude in
//          [2^13, 2^14); hi = fp16(s x), lo = fp16(s x - hi).  hi and lo carry 22 significant
//          bits, so hi*hi + hi*lo + lo*hi is accurate to about 2^-21 relative.
// A left operand is laid out [hi | hi | lo] along K, a right one [hi | lo | hi] (pattern b), each
// part K' (K rounded up to 64) wide; the single-pass form keeps [hi] alone.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace gvt {
namespace split16 {

__device__ __forceinline__ void split8_bf16(const float (&x)[8], uint4& hi, uint4& lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * e] - hf.x, x[2 * e + 1] - hf.y);
        h[e] = *reinterpret_cast<const uint32_t*>(&hb);
        l[e] = *reinterpret_cast<const uint32_t*>(&lb);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void split8_f16(const float (&x)[8], float s, uint4& hi, uint4& lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float a = x[2 * e] * s, b = x[2 * e + 1] * s;
        const __half2 hh = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(hh);
        const __half2 lh = __floats2half2_rn(a - hf.x, b - hf.y);
        h[e] = *reinterpret_cast<const uint32_t*>(&hh);
        l[e] = *reinterpret_cast<const uint32_t*>(&lh);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// power-of-two scale putting amax in [2^13, 2^14); 1 for zero or non-finite rows
__device__ __forceinline__ void row_scale(float amax, float& s, float& inv)
{
    if (!(amax > 0.f) || !isfinite(amax)) {
        s = 1.f;
        inv = 1.f;
        return;
    }
    int e;
    frexpf(amax, &e);   // amax = f 2^e, f in [0.5, 1)
    e = max(e, -100);
    s = ldexpf(1.f, 14 - e);
    inv = ldexpf(1.f, e - 14);
}

// the `parts` copies of one 8-value group q of a row, per_row groups apart
__device__ __forceinline__ void store3(uint4* d, int64_t q, int64_t per_row, int pattern_b, int parts,
                                       const uint4& hi, const uint4& lo)
{
    d[q] = hi;
    if (parts == 1) return;
    d[per_row + q] = pattern_b ? lo : hi;
    d[2 * per_row + q] = pattern_b ? hi : lo;
}

}  // namespace split16
}  // namespace gvt
