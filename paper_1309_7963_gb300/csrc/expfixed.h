// e^x in double precision for a float argument x, on the integer pipes: GB300's FP64 pipe
// runs at 1/64 of the FP32 rate, and the FP32 mode's evaporation widths take one exponential
// each. The method is the table-driven exponential of Tang (ACM Trans. Math. Softw. 15 (1989)
// 144) in fixed point:
//   y = x log2(e), exact to 2^-86 (x is m 2^(E-23) exactly; log2(e) to 96 bits);
//   e^x = 2^k 2^(j/64) e^r, k = floor(y), j the next 6 bits of y, r = (the remaining bits of
//   y) ln 2 < ln(2)/64;
//   e^r = 1 + r (1 + r (1/2 + r (1/6 + ... r/7!))) by Horner in Q1.63 (64-bit words, value
//   times 2^63), with its truncation below 2^-66;
//   2^(j/64) from a table in Q1.63 (rounded to nearest);
//   the product (in [1, 2), Q2.62) rounded to 53 bits, to nearest with ties to even, and
//   assembled with the exponent k.
// Every step keeps at least 61 correct bits, so the result is within 0.51 ulp of e^x (the
// correctly rounded double for all but about 1 argument in 1000). Arguments in [1, 256);
// the FP32 mode's widths take x = 2 sqrt(aY) <= 200 for every nucleus the library accepts.
#pragma once

#include <cstdint>

namespace pnuc {
namespace dev {
namespace {

constexpr uint64_t kLog2eHi = 0xB8AA3B295C17F0BBull, kLog2eLo = 0xBE87FED0ull;  // log2(e) 2^95
constexpr uint64_t kLn2Q64 = 0xB17217F7D1CF79ACull;                             // ln(2) 2^64
// 2^(j/64) 2^63, j = 0..63
__device__ const uint64_t kExp2Q63[64] = {
    0x8000000000000000ull, 0x8164D1F3BC030773ull, 0x82CD8698AC2BA1D7ull, 0x843A28C3ACDE4046ull,
    0x85AAC367CC487B15ull, 0x871F61969E8D1010ull, 0x88980E8092DA8527ull, 0x8A14D575496EFD9Aull,
    0x8B95C1E3EA8BD6E7ull, 0x8D1ADF5B7E5BA9E6ull, 0x8EA4398B45CD53C0ull, 0x9031DC431466B1DCull,
    0x91C3D373AB11C336ull, 0x935A2B2F13E6E92Cull, 0x94F4EFA8FEF70961ull, 0x96942D3720185A00ull,
    0x9837F0518DB8A96Full, 0x99E0459320B7FA65ull, 0x9B8D39B9D54E5539ull, 0x9D3ED9A72CFFB751ull,
    0x9EF5326091A111AEull, 0xA0B0510FB9714FC2ull, 0xA27043030C496819ull, 0xA43515AE09E6809Eull,
    0xA5FED6A9B15138EAull, 0xA7CD93B4E965356Aull, 0xA9A15AB4EA7C0EF8ull, 0xAB7A39B5A93ED337ull,
    0xAD583EEA42A14AC6ull, 0xAF3B78AD690A4375ull, 0xB123F581D2AC2590ull, 0xB311C412A9112489ull,
    0xB504F333F9DE6484ull, 0xB6FD91E328D17791ull, 0xB8FBAF4762FB9EE9ull, 0xBAFF5AB2133E45FBull,
    0xBD08A39F580C36BFull, 0xBF1799B67A731083ull, 0xC12C4CCA66709456ull, 0xC346CCDA24976407ull,
    0xC5672A115506DADDull, 0xC78D74C8ABB9B15Dull, 0xC9B9BD866E2F27A3ull, 0xCBEC14FEF2727C5Dull,
    0xCE248C151F8480E4ull, 0xD06333DAEF2B2595ull, 0xD2A81D91F12AE45Aull, 0xD4F35AABCFEDFA1Full,
    0xD744FCCAD69D6AF4ull, 0xD99D15C278AFD7B6ull, 0xDBFBB797DAF23755ull, 0xDE60F4825E0E9124ull,
    0xE0CCDEEC2A94E111ull, 0xE33F8972BE8A5A51ull, 0xE5B906E77C8348A8ull, 0xE8396A503C4BDC68ull,
    0xEAC0C6E7DD24392Full, 0xED4F301ED9942B84ull, 0xEFE4B99BDCDAF5CBull, 0xF281773C59FFB13Aull,
    0xF5257D152486CC2Cull, 0xF7D0DF730AD13BB9ull, 0xFA83B2DB722A033Aull, 0xFD3E0C0CF486C175ull};

__device__ __forceinline__ double exp_fixed(float x)
{
    // 1/n! 2^63, n = 1..7
    constexpr uint64_t kInvFact[7] = {0x8000000000000000ull, 0x4000000000000000ull, 0x1555555555555555ull,
                                      0x0555555555555555ull, 0x0111111111111111ull, 0x002D82D82D82D82Eull,
                                      0x0006806806806807ull};
    const uint32_t u = __float_as_uint(x);
    const int E = (int)(u >> 23) - 127;  // 0 .. 7 for x in [1, 256)
    const uint64_t X = (uint64_t)((u & 0x7FFFFFu) | 0x800000u) << E;  // x 2^23, < 2^31
    // P = X (kLog2eHi 2^32 + kLog2eLo) / 2^32 = y 2^86, as hi:lo (the low product truncated)
    uint64_t lo = X * kLog2eHi, hi = __umul64hi(X, kLog2eHi);
    const uint64_t t = (X * kLog2eLo) >> 32;
    lo += t;
    hi += lo < t ? 1u : 0u;
    const int k = (int)(hi >> 22);
    const uint64_t f = (hi << 42) | (lo >> 22);  // the fraction of y, Q0.64
    const int j = (int)(f >> 58);
    const uint64_t r = __umul64hi(f & ((1ull << 58) - 1u), kLn2Q64);  // Q0.64, < ln(2)/64
    uint64_t s = kInvFact[6];
#pragma unroll
    for (int n = 5; n >= 0; --n) s = kInvFact[n] + __umul64hi(r, s);
    const uint64_t er = (1ull << 63) + __umul64hi(r, s);       // e^r, Q1.63
    const uint64_t M = __umul64hi(__ldg(&kExp2Q63[j]), er);   // 2^(j/64) e^r, Q2.62, in [2^62, 2^63)
    uint64_t q = M >> 10;
    const uint32_t rem = (uint32_t)M & 0x3FFu;
    q += (rem > 512u || (rem == 512u && (q & 1u))) ? 1u : 0u;
    const int ke = q >> 53 ? k + 1 : k;  // rounding carried into the next binade
    q = q >> 53 ? q >> 1 : q;
    return __longlong_as_double((long long)(((uint64_t)(ke + 1023) << 52) | (q - (1ull << 52))));
}

}  // namespace
}  // namespace dev
}  // namespace pnuc
