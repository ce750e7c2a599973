// SNES draws (Sec. II.E, Eq. 35): standard normals from the counter-based
// generator Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11), written
// from its published definition, and the Box-Muller transform.  Element e of
// the draws of generation `gen` comes from block e / 4 with counter
// {e / 4, 0, gen, 0x4E4550} and key {seed lo, seed hi}; u = (w + 1/2) 2^-32;
// lanes 0/1 (2/3) are the Box-Muller pair of (u0, u1) ((u2, u3)).  Both the
// draw kernel and the packing kernel that draws while it packs use these
// functions, so that they give the same bits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nep {

__device__ __forceinline__ void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                                       uint32_t (&o)[4])
{
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    o[0] = c0;
    o[1] = c1;
    o[2] = c2;
    o[3] = c3;
}

// u = (w + 1/2) 2^-32 rounded once to FP32 (round to nearest), from 32-bit
// integer conversions (the FP64 pipe is slow on this part).  Below 2^31,
// 2 w + 1 fits 32 bits and converts exactly-rounded.  From 2^31 on, FP32
// values are 256 apart there and w + 1/2 is never halfway between two of
// them, so its rounding is that of w except where w itself is halfway
// (w = 128 mod 256), where ties-to-even may round w down but w + 1/2 rounds
// up.
__device__ __forceinline__ float unit_from_word(uint32_t w)
{
    if (w < 0x80000000u) return __uint2float_rn(2u * w + 1u) * 0x1p-33f;
    const float a = (w & 255u) == 128u ? __uint2float_ru(w) : __uint2float_rn(w);
    return a * 0x1p-32f;
}

// The Box-Muller pair of two 32-bit words, u = (w + 1/2) 2^-32: the transform
// runs in FP32 with ln u0 taken as log1p(-(1 - u0)) when u0 >= 1/2 (1 - u0 =
// (~w0 + 1/2) 2^-32 exactly), so that the radius keeps full relative
// precision where ln u0 is tiny.
__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float& g0, float& g1)
{
    const float lu = w0 < 0x80000000u ? logf(unit_from_word(w0)) : log1pf(-unit_from_word(~w0));
    const float rad = sqrtf(-2.f * lu);
    float sn, cs;
    sincospif(2.f * unit_from_word(w1), &sn, &cs);
    g0 = rad * cs;
    g1 = rad * sn;
}

// The four words of Philox block b of the stream (seed, gen).
__device__ __forceinline__ void philox_block(long long b, unsigned gen, unsigned long long seed, uint32_t (&w)[4])
{
    philox((uint32_t)b, 0u, gen, 0x4E4550u, (uint32_t)seed, (uint32_t)(seed >> 32), w);
}

// Element e of the stream alone (one block, the pair that holds it).
__device__ __forceinline__ float normal_at(long long e, unsigned gen, unsigned long long seed)
{
    uint32_t w[4];
    philox_block(e >> 2, gen, seed, w);
    const int l = (int)(e & 3), pr = l >> 1;
    float g0, g1;
    box_muller(w[2 * pr], w[2 * pr + 1], g0, g1);
    return (l & 1) ? g1 : g0;
}

}  // namespace nep
