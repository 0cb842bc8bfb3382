// bits.cuh: exact FP64 helpers on the integer pipe, shared by the kernel
// translation units. On this GPU the FP64 unit issues one warp instruction
// per 64 cycles per SM sub-partition, and FP64 comparisons, min, max and
// the FP32 <-> FP64 conversion instructions all issue on it, so work that
// is exact on the bits (doublings, sign tests, order tests, widenings,
// roundings) is done with integer instructions instead.
//
// Not a standalone header: each translation unit includes it inside its own
// namespace.
#ifndef OPF_BITS_CUH
#define OPF_BITS_CUH

// 2 v exactly, on the integer pipe: a normal v gets one more in its exponent
// field; zero and subnormals shift their magnitude left by one (carrying into
// the exponent field where the result becomes normal); the largest binade
// overflows to infinity; infinities and NaNs are returned unchanged.
__device__ __forceinline__ double twice(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned long long sign = b & 0x8000000000000000ULL;
    const unsigned long long mag = b & 0x7fffffffffffffffULL;
    const unsigned ex = (unsigned)(mag >> 52);
    unsigned long long r = b + (1ULL << 52);
    r = ex == 0u ? (sign | (mag << 1)) : r;
    r = ex == 0x7feu ? (sign | 0x7ff0000000000000ULL) : r;
    r = ex == 0x7ffu ? b : r;
    return __longlong_as_double((long long)r);
}

// a 64-bit integer key in the order of the doubles (NaN excepted; -0 sorts
// just below +0)
__device__ __forceinline__ long long order_key(double x)
{
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : b ^ 0x7FFFFFFFFFFFFFFFll;
}

// x - clip(x, -h, h) for h >= 0: 0 inside (no FP64 instruction), one
// subtraction outside, its sign from the sign bit; a NaN x stays NaN
__device__ __forceinline__ double excess_sym(double x, double h)
{
    const long long bx = __double_as_longlong(x);
    if ((bx & 0x7FFFFFFFFFFFFFFFll) <= __double_as_longlong(h))
        return 0.0;
    return bx >= 0 ? x - h : x + h;
}

// x is +0 or -0 (an integer test)
__device__ __forceinline__ bool is_zero(double x)
{
    return ((unsigned long long)__double_as_longlong(x) << 1) == 0ULL;
}

// x rounded to the nearest FP32 (ties to even); the conversion instruction
// is kept for the values outside FP32's normal range only (zero and double
// subnormals round to a signed zero exactly)
__device__ __forceinline__ float f32_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0)
        return __uint_as_float(sign);
    const int ef = e - 1023 + 127;  // FP32 biased exponent
    if (ef <= 0 || ef >= 255)
        return (float)x;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;  // 52 fraction bits
    const unsigned int mf = (unsigned int)(m >> 29);        // the 23 kept
    const unsigned long long rem = m & 0x1FFFFFFFull, half = 1ull << 28;
    unsigned int bits = ((unsigned int)ef << 23) | mf;
    if (rem > half || (rem == half && (mf & 1u)))
        bits += 1u;  // a carry moves into the exponent (to infinity past the largest float)
    return __uint_as_float(bits | sign);
}

// f exactly as a double: normal values and zeros on the integer pipe, the
// rest (subnormals, infinities, NaN) by the conversion instruction
__device__ __forceinline__ double widen(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned ex = (b >> 23) & 0xffu;
    if (ex == 0u && (b & 0x7fffffu) == 0u)
        return __longlong_as_double((long long)(b & 0x80000000u) << 32);  // +-0
    if (ex == 0u || ex == 0xffu)
        return (double)f;
    const unsigned hi = (b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

#endif
