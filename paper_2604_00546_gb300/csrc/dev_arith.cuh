// Device-side 64-bit RNS arithmetic for sm_103a.
//
// Residues are kept canonical ([0, q)) between kernels. Products by constants
// use Shoup's precomputed quotient (w' = floor(w * 2^64 / q)); products of two
// variable residues and multiply-accumulate chains use Montgomery reduction
// with R = 2^64 (one operand stored pre-multiplied by R, or a second
// reduction by R^2 mod q). All primes are below 2^61, which the lazy
// accumulation bounds below rely on.
#pragma once
#include <cstdint>

typedef uint64_t u64;
typedef unsigned int u32;

struct DevPrime {
    u64 q;       // modulus
    u64 qinv;    // q^-1 mod 2^64 (Montgomery)
    u64 r2;      // 2^128 mod q
    u64 ninv;    // N^-1 mod q
    u64 ninv_s;  // Shoup quotient of ninv
    u64 one_s;   // floor(2^64 / q): Shoup quotient of 1 (x mod q for any 64-bit x)
};

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// x * w mod q for a constant w with Shoup quotient ws; any 64-bit x.
__device__ __forceinline__ u64 mul_shoup(u64 x, u64 w, u64 ws, u64 q) {
    u64 hi = __umul64hi(x, ws);
    u64 r = x * w - hi * q;
    return r >= q ? r - q : r;
}

// Montgomery reduction of T = hi * 2^64 + lo with hi < q: returns T * 2^-64 mod q in [0, q).
__device__ __forceinline__ u64 redc(u64 hi, u64 lo, u64 q, u64 qinv) {
    u64 m = lo * qinv;
    u64 t = __umul64hi(m, q);
    return hi >= t ? hi - t : hi - t + q;
}

struct Acc128 {
    u64 lo, hi;
};
__device__ __forceinline__ void mac128(Acc128& a, u64 x, u64 y) {
    u64 l = x * y;
    u64 h = __umul64hi(x, y);
    a.lo += l;
    a.hi += h + (a.lo < l ? 1ull : 0ull);
}

// Products of residues below 2^60 from 30-bit halves: x = xh 2^30 + xl, y = yh 2^30 + yl,
// x y = xl yl + (xl yh + xh yl) 2^30 + xh yh 2^60. Each partial product is below 2^60, so up
// to 8 products sum in three 64-bit words, a1 holding the middle terms (below 2^64), with no
// carries. split30 packs (xl, xh) into the low and high 32-bit words.
struct Acc3 {
    u64 a0, a1, a2;
};
__device__ __forceinline__ u64 split30(u64 x) { return (x & 0x3fffffffull) | ((x >> 30) << 32); }
// acc += hi 2^64 + lo, one add-with-carry chain
__device__ __forceinline__ void add128(Acc128& acc, u64 lo, u64 hi) {
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(acc.lo), "+l"(acc.hi) : "l"(lo), "l"(hi));
}
// acc += a0 + a1 2^30 + a2 2^60, then a = 0
__device__ __forceinline__ void flush30(Acc128& acc, Acc3& a) {
    add128(acc, a.a0, 0);
    add128(acc, a.a1 << 30, a.a1 >> 34);
    add128(acc, a.a2 << 60, a.a2 >> 4);
    a.a0 = a.a1 = a.a2 = 0;
}

// Karatsuba form of the same sums, three multiply-adds per product:
//   x y = xl yl + ((xl + xh)(yl + yh) - xl yl - xh yh) 2^30 + xh yh 2^60.
// am = sum (xl + xh)(yl + yh) may wrap modulo 2^64, but the middle term sum (xl yh + xh yl) is
// below 8 * 2 * 2^60 = 2^64 for up to 8 products, so am - a0 - a2 modulo 2^64 is exact.
// xsum = xl + xh is passed in (it is shared by every product with the same x).
struct AccK {
    u64 a0, am, a2;
};
__device__ __forceinline__ u32 sum30(u64 xs) { return (u32)xs + (u32)(xs >> 32); }
__device__ __forceinline__ void mack(AccK& a, u64 xs, u32 xsum, u64 ys) {
    const u32 xl = (u32)xs, xh = (u32)(xs >> 32), yl = (u32)ys, yh = (u32)(ys >> 32);
    a.a0 += (u64)xl * yl;
    a.am += (u64)xsum * (yl + yh);
    a.a2 += (u64)xh * yh;
}
// acc += the products summed in a, then a = 0
__device__ __forceinline__ void flushk(Acc128& acc, AccK& a) {
    Acc3 t{a.a0, a.am - a.a0 - a.a2, a.a2};
    flush30(acc, t);
    a.a0 = a.am = a.a2 = 0;
}

// a * b mod q for two variable residues: REDC(REDC(a b) * R^2)
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const DevPrime& P) {
    u64 t = redc(__umul64hi(a, b), a * b, P.q, P.qinv);
    return redc(__umul64hi(t, P.r2), t * P.r2, P.q, P.qinv);
}

// x * R mod q (Montgomery form)
__device__ __forceinline__ u64 to_mont(u64 x, const DevPrime& P) {
    return redc(__umul64hi(x, P.r2), x * P.r2, P.q, P.qinv);
}

// Automorphism sigma_g in evaluation form: position k holds the value at
// psi^(2 brev(k) + 1); sigma_g(a) at that point is a at psi^((2 brev(k)+1) g).
__device__ __forceinline__ u32 galois_src_index(u32 k, u32 g, int logN) {
    u32 e = 2u * (__brev(k) >> (32 - logN)) + 1u;
    u32 M = 2u << logN;
    u32 e2 = (u32)(((u64)e * g) & (M - 1));
    return __brev((e2 - 1u) >> 1) >> (32 - logN);
}
