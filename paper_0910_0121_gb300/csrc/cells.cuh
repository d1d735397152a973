// The finest-cell index of a coordinate (reading C9 of the key, Sec. 3.2.5): the
// periodic wrap into [0, L), then floor((r/L) 2^21) clamped to [0, 2^21-1], in exact
// IEEE FP64 steps (no fused multiply-add) or, for a power-of-two L, by integer
// operations on the bits.  Shared by the key kernel and the domain kernels, so that a
// particle's cell is the same wherever it is computed.
#pragma once
#include "common.cuh"

namespace greem {

// floor((r/L) 2^21) clamped to [0, 2^21-1].  r * (1/L) differs from the rounded
// quotient by at most 3 ulp, i.e. by < 1e-9 after the scaling, so its floor is the same
// unless the scaled value lies within 1e-6 of an integer; only then is the exact
// quotient formed.
__device__ __forceinline__ uint32_t cell21(double r, double L, double invL)
{
    double q = __dmul_rn(__dmul_rn(r, invL), 2097152.0);
    double f = floor(q);
    const double fr = q - f;
    if (fr < 1e-6 || fr > 1.0 - 1e-6) f = floor(__dmul_rn(__ddiv_rn(r, L), 2097152.0));
    long long i = (long long)f;
    i = i < 0 ? 0 : i;
    i = i > 2097151 ? 2097151 : i;
    return (uint32_t)i;
}

// Power-of-two box side (the usual L = 1): (r/L) 2^21 = r 2^(21-e) exactly, so the cell
// index is read from the bits of r with integer operations only (no FP64 pipe work).
// Same result as cell21(): the quotient is exact, and floor of the scaled value is the
// integer part of the binary expansion.
__device__ __forceinline__ uint32_t cell21_pow2(double r, int e)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(r);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;  // zero or subnormal
    const unsigned long long mant = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = (ex - 1023) - 52 + 21 - e;  // value = mant * 2^sh
    long long i;
    if (sh >= 0) i = sh >= 11 ? (1ll << 62) : (long long)(mant << sh);
    else i = -sh >= 64 ? 0 : (long long)(mant >> (-sh));
    i = i > 2097151 ? 2097151 : i;
    return (uint32_t)i;
}

// The general-L cell indices as a real call: inlined, the compiler may predicate its
// FP64 work into the lanes of the power-of-two path, where it still occupies the FP64
// pipe.
static __device__ __noinline__ uint3 cells_general(double x, double y, double z, double L, double invL)
{
    return make_uint3(cell21(wrap_pos_fast(x, L), L, invL), cell21(wrap_pos_fast(y, L), L, invL),
                      cell21(wrap_pos_fast(z, L), L, invL));
}

// The three finest-cell indices of a position (the key's cells, reading C9).
__device__ __forceinline__ uint3 cells_of(double x, double y, double z, double L, double invL, int pow2_e)
{
    if (pow2_e != kNotPow2)
        return make_uint3(cell21_pow2(wrap_pos_fast(x, L), pow2_e), cell21_pow2(wrap_pos_fast(y, L), pow2_e),
                          cell21_pow2(wrap_pos_fast(z, L), pow2_e));
    return cells_general(x, y, z, L, invL);
}

}  // namespace greem
