// gcmc_device.cuh -- device-side building blocks of the GCMC hot path:
// counter-based random numbers, grid/cell arithmetic and the Lennard-Jones
// pair term (Eq. 1) in FP32 and FP64.  Included by every kernel file.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gcmc {

constexpr int kMaxSpecies = 8;
constexpr int kWarp = 32;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, each two 32x32->64-bit
// multiplies whose halves are mixed with the other counter words and the
// key; the key advances by the two Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct Words8 {
    uint32_t w[8];
};

__device__ __forceinline__ uint4 philox_block(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a0 = 0xD2511F53u * c.x;  // low half of M0 * c0
        const uint32_t h0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t a1 = 0xCD9E8D57u * c.z;  // low half of M1 * c2
        const uint32_t h1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(h1 ^ c.y ^ k.x, a1, h0 ^ c.w ^ k.y, a0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// The eight words of move m of chain `chain`.
__device__ __forceinline__ Words8 move_words(uint64_t seed, uint64_t m, uint32_t chain)
{
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint4 a = philox_block(make_uint4((uint32_t)m, (uint32_t)(m >> 32), chain, 0u), key);
    const uint4 b = philox_block(make_uint4((uint32_t)m, (uint32_t)(m >> 32), chain, 1u), key);
    Words8 r;
    r.w[0] = a.x; r.w[1] = a.y; r.w[2] = a.z; r.w[3] = a.w;
    r.w[4] = b.x; r.w[5] = b.y; r.w[6] = b.z; r.w[7] = b.w;
    return r;
}

// 53-bit uniform in [0, 1) from words 6 and 7.
__device__ __forceinline__ double uniform53(uint32_t w6, uint32_t w7)
{
    const uint64_t k = ((uint64_t)(w6 >> 5) << 26) | (uint64_t)(w7 >> 6);
    return (double)k * 1.1102230246251565404e-16;  // 2^-53
}

// The index a displacement (type 0) or a deletion (type 2) picks among n >= 1
// candidates (Algorithm 1's uniform choice): 2^k the smallest power of two at
// least n, the top k bits of the tries -- w[1], w[2], w[3] for a deletion;
// w[1] and, for k <= 16, the top k bits of w[1]'s low half for a
// displacement -- and the first one below n wins (rejection sampling);
// when none does, floor(f n / 2^32) of f = w[4] (deletion) or w[5]
// (displacement), words independent of the tries.  The index moves with n
// only when n passes a power of two, when a try lies between the two
// counts, or when every try fails, so a speculative evaluation that guessed
// the count slightly wrong usually picked the right particle all the same.
__device__ __forceinline__ int pick_index(uint32_t n, const uint32_t *w, int type)
{
    const int k = 32 - __clz((int)(n - 1u));  // n = 1: clz(0) = 32, k = 0
    if (k == 0) return 0;
    const int sh = 32 - k;
    uint32_t d = w[1] >> sh;
    if (d < n) return (int)d;
    if (type == 2) {
        d = w[2] >> sh;
        if (d < n) return (int)d;
        d = w[3] >> sh;
        if (d < n) return (int)d;
        return (int)__umulhi(w[4], n);
    }
    if (k <= 16) {
        d = (w[1] << 16) >> sh;
        if (d < n) return (int)d;
    }
    return (int)__umulhi(w[5], n);
}

// Whether pick_index gives the same index for every count in [lo, hi]
// (1 <= lo <= hi): the counts share k, and a try below lo comes before any
// try in [lo, hi).
__device__ __forceinline__ bool pick_is_stable(uint32_t lo, uint32_t hi, const uint32_t *w, int type)
{
    const int k = 32 - __clz((int)(hi - 1u));
    if (32 - __clz((int)(lo - 1u)) != k) return false;
    if (k == 0) return true;
    const int sh = 32 - k;
    uint32_t tries[3];
    int nt = 1;
    tries[0] = w[1] >> sh;
    if (type == 2) {
        tries[1] = w[2] >> sh;
        tries[2] = w[3] >> sh;
        nt = 3;
    } else if (k <= 16) {
        tries[1] = (w[1] << 16) >> sh;
        nt = 2;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j < nt) {
            if (tries[j] < lo) return true;
            if (tries[j] < hi) return false;
        }
    }
    return false;  // every try fails for some count: the fallback depends on it
}

// ---------------------------------------------------------------------------
// Grid and cells
// ---------------------------------------------------------------------------
// The grid coordinate of x (Sec. 3.2.1's binning on the 2^32 grid):
// floor(x q) wrapped to 32 bits.  ok turns false when x q is not finite or
// |x q| > 4e18.  One FP64 multiply and one conversion that rounds down (the
// FP64 pipe is narrow on this part); the range test compares the magnitude's
// bit pattern, which orders like the value.
__device__ __forceinline__ uint32_t quantize_axis(double x, double q, bool &ok)
{
    const double t = x * q;
    const unsigned long long mag = (unsigned long long)__double_as_longlong(t) & 0x7fffffffffffffffull;
    if (mag > 0x43cbc16d674ec800ull) {  // the bits of 4e18; NaN and infinities are above
        ok = false;
        return 0u;
    }
    return (uint32_t)(unsigned long long)__double2ll_rd(t);
}

// floor(X * T / 2^32): the cell coordinate of grid coordinate X.
__device__ __forceinline__ int cell_coord(uint32_t X, uint32_t T) { return (int)__umulhi(X, T); }

__device__ __forceinline__ int cell_of(uint32_t X, uint32_t Y, uint32_t Z, int T)
{
    return (cell_coord(Z, (uint32_t)T) * T + cell_coord(Y, (uint32_t)T)) * T +
           cell_coord(X, (uint32_t)T);
}

// Cell id of the neighbour at offset (ox, oy, oz) in {-1,0,1}^3.
__device__ __forceinline__ int neighbour_cell(int cx, int cy, int cz, int k, int T)
{
    int ox = k % 3 - 1, oy = (k / 3) % 3 - 1, oz = k / 9 - 1;
    int nx = cx + ox, ny = cy + oy, nz = cz + oz;
    nx += (nx < 0) ? T : 0;
    nx -= (nx >= T) ? T : 0;
    ny += (ny < 0) ? T : 0;
    ny -= (ny >= T) ? T : 0;
    nz += (nz < 0) ? T : 0;
    nz -= (nz >= T) ? T : 0;
    return (nz * T + ny) * T + nx;
}

// Particle tag stored in the 4th word of a position: (index << 8) | species.
__device__ __forceinline__ uint32_t make_tag(uint32_t i, uint32_t s) { return (i << 8) | s; }
__device__ __forceinline__ uint32_t tag_species(uint32_t t) { return t & 0xFFu; }
__device__ __forceinline__ uint32_t tag_index(uint32_t t) { return t >> 8; }

// Exact squared grid distance of the minimum image (the uint32 difference
// reinterpreted as int32 is the periodic image nearest to zero).
struct GridSep {
    int dx, dy, dz;
    unsigned long long g;
};

__device__ __forceinline__ GridSep grid_sep(uint4 a, uint4 b)
{
    GridSep s;
    s.dx = (int)(a.x - b.x);
    s.dy = (int)(a.y - b.y);
    s.dz = (int)(a.z - b.z);
    s.g = (unsigned long long)((long long)s.dx * s.dx) + (unsigned long long)((long long)s.dy * s.dy) +
          (unsigned long long)((long long)s.dz * s.dz);
    return s;
}

// ---------------------------------------------------------------------------
// Force-field constants, per species pair, in grid units:
//   c4e = 4 eps,  sig2 = (sigma / h)^2,
//   U = c4e (s^6 s^6 - s^6) with s^2 = sig2 / r_grid^2.
// ---------------------------------------------------------------------------
struct FieldF {
    float c4e[kMaxSpecies * kMaxSpecies];
    float sig2[kMaxSpecies * kMaxSpecies];
    // the rounding residues: c4e + c4e_lo and sig2 + sig2_lo are the FP64
    // constants to about 2^-48 (the compensated pair term below uses them)
    float c4e_lo[kMaxSpecies * kMaxSpecies];
    float sig2_lo[kMaxSpecies * kMaxSpecies];
};
struct FieldD {
    double c4e[kMaxSpecies * kMaxSpecies];
    double sig2[kMaxSpecies * kMaxSpecies];
};

// Pair energy in FP32 from an exact grid separation known to be inside the
// cutoff.  rep/att are the two terms' magnitudes.
__device__ __forceinline__ void lj_f32(const GridSep &s, float c4e, float sig2, float &u, float &mag)
{
    const float fx = (float)s.dx, fy = (float)s.dy, fz = (float)s.dz;
    const float r2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
    const float s2 = sig2 / r2;
    const float s6 = s2 * s2 * s2;
    const float rep = c4e * s6 * s6;
    const float att = c4e * s6;
    u = rep - att;
    mag = rep + att;
    if (s.g == 0ull) {
        u = __int_as_float(0x7f800000);
        mag = u;
    }
}

// Compensated FP32 pair energy (float-float, after Dekker's double-length
// arithmetic, Numer. Math. 18 (1971): a value is an unevaluated sum hi + lo
// of two floats; TwoProduct takes the exact rounding error of a product with
// one FMA, TwoSum (Knuth) the exact error of a sum).  From the exact integer
// separation (ex, ey, ez) of a pair inside the cutoff:
//   r^2 = g exactly as an integer, split into r2h + r2l;
//   s^2 = sig2 / r^2: an approximate quotient q corrected by its residual;
//   s^6 = (s^2)^3, t = s^6 - 1, v = s^6 t, U = c4e v, each step keeping its
//   rounding error in the low word.
// Every operation is FP32 (the FP32 pipe); the result uh + ul carries a
// relative error near 1e-13 of rep + att, where a plain FP32 evaluation
// carries about 1e-6.  m = rep + att in plain FP32 (an error scale only).
// g == 0 (both particles on one grid point) gives U = +inf.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// g (< 2^63) as a float-float hi + lo, with 32-bit conversions and integer
// operations only (64-bit integer conversions run on the FP64 pipe, a small
// fraction of the FP32 one): hi approximates g, the integer value of hi is
// rebuilt from its bits, and the exact remainder g - hi (|r| < 2^40) is
// converted as (r >> 16) * 2^16 + (r & 0xFFFF), both parts exact in FP32.
__device__ __forceinline__ void split_u64(unsigned long long g, float &hi, float &lo)
{
    const uint32_t gh = (uint32_t)(g >> 32), gl = (uint32_t)g;
    hi = fmaf(__uint2float_rn(gh), 4294967296.0f, __uint2float_rn(gl));
    // the integer value of hi: mantissa shifted by its exponent
    const uint32_t bits = __float_as_uint(hi);
    const int ex = (int)(bits >> 23) - 150;  // hi = mant * 2^ex
    const unsigned long long mant = (unsigned long long)((bits & 0x7FFFFFu) | 0x800000u);
    const unsigned long long hv = ex >= 0 ? (mant << ex) : (mant >> -ex);
    const long long r = (long long)(g - hv);
    lo = fmaf(__int2float_rn((int)(r >> 16)), 65536.0f, __uint2float_rn((uint32_t)r & 0xFFFFu));
}

__device__ __forceinline__ void lj_ff(int ex, int ey, int ez, float ch, float cl, float sh, float sl, float &uh,
                                      float &ul, float &m)
{
    const unsigned long long g = (unsigned long long)((long long)ex * ex) +
                                 (unsigned long long)((long long)ey * ey) +
                                 (unsigned long long)((long long)ez * ez);
    if (g == 0ull) {
        uh = __int_as_float(0x7f800000);
        ul = 0.f;
        m = uh;
        return;
    }
    float r2h, r2l;
    split_u64(g, r2h, r2l);
    const float rcp = rcp_approx(r2h);
    // s^2 = q + ql: the residual (sh + sl) - q (r2h + r2l) divided by r^2
    const float q = __fmul_rn(sh, rcp);
    float res = fmaf(-q, r2h, sh);
    res = fmaf(-q, r2l, __fadd_rn(res, sl));
    const float ql = __fmul_rn(res, rcp);
    // s^6 = (q + ql)^3 = q^3 + 3 q^2 ql + ...: the two products exactly
    const float a = __fmul_rn(q, q), ae = fmaf(q, q, -a);
    const float b = __fmul_rn(a, q), be = fmaf(a, q, -b);
    const float s6l = fmaf(__fmul_rn(3.f, a), ql, fmaf(ae, q, be));
    // t = s^6 - 1 (TwoSum of b and -1)
    const float t = __fadd_rn(b, -1.f);
    const float bb = __fsub_rn(t, b);
    const float te = __fadd_rn(__fsub_rn(b, __fsub_rn(t, bb)), __fsub_rn(-1.f, bb));
    const float tl = __fadd_rn(te, s6l);
    // v = s^6 (s^6 - 1)
    const float vh = __fmul_rn(b, t);
    const float vl = fmaf(b, tl, fmaf(s6l, t, fmaf(b, t, -vh)));
    // U = c4e v
    uh = __fmul_rn(ch, vh);
    ul = fmaf(ch, vl, fmaf(cl, vh, fmaf(ch, vh, -uh)));
    m = ch * b * (b + 1.f);
}

// hi + lo += x_hi + x_lo for a running sum of few terms: TwoSum on the high
// words, the low words and the error summed in FP32.
__device__ __forceinline__ void ff_acc(float &hi, float &lo, float xh, float xl)
{
    const float s = __fadd_rn(hi, xh);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(xh, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, xl));
}

__device__ __forceinline__ void lj_f64(const GridSep &s, double c4e, double sig2, double &u,
                                       double &mag)
{
    const double fx = (double)s.dx, fy = (double)s.dy, fz = (double)s.dz;
    const double r2 = fx * fx + fy * fy + fz * fz;
    const double s2 = sig2 / r2;
    const double s6 = s2 * s2 * s2;
    const double rep = c4e * s6 * s6;
    const double att = c4e * s6;
    u = rep - att;
    mag = rep + att;
    if (s.g == 0ull) {
        u = __longlong_as_double(0x7ff0000000000000ll);
        mag = u;
    }
}

// Float-float values (hi + lo) and their sums (TwoSum on the high words).
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    const float t = e + a.lo + b.lo;
    const float h = s + t;
    return FF{h, t - (h - s)};
}
__device__ __forceinline__ FF ff_add_f(FF a, float x)
{
    const float s = a.hi + x;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (x - bb);
    const float t = e + a.lo;
    const float h = s + t;
    return FF{h, t - (h - s)};
}
__device__ __forceinline__ FF ff_warp_sum(FF v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FF w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = ff_add(v, w);
    }
    return v;
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_inclusive_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Device status word bits.
enum : int {
    kStatusCellOverflow = 1,
    kStatusCapacity = 2,
    kStatusNonFinite = 4,
    kStatusBadInput = 8,
    kStatusTimeout = 16,
};

}  // namespace gcmc
