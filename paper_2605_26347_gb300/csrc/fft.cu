// The oversampled 2-D DFT F of Eq. 6 and its adjoint, as four row passes.
//
// Forward, for w-bin p (F Z_p of Eq. 6):
//   rows pass  : image row i (n_x pixels) -> z = x * Z_p (grid correction and the w-layer
//                chirp, Section 3.2) -> zero-padded 2n_x-point DFT along l, written
//                transposed as A^T[u][i]  (2 n_x rows of n_y).
//   cols pass  : row u of A^T -> zero-padded 2n_y-point DFT along m -> X[u][v].
// Adjoint (Z_p^dagger F^dagger of Eq. 8):
//   cols pass  : row u of Xh (2 n_y cells) -> 2n_y-point inverse DFT cropped to the n_y
//                image rows -> B[i][u], transposed.
//   rows pass  : row i of B (2 n_x cells) -> cropped inverse DFT along u -> * conj(Z_p),
//                accumulated into the output image.
//
// Each pass is one 2N-point Stockham radix-16 FFT per row held in registers (16 points per
// thread, 2N/16 threads per row), exchanging through shared memory between stages; at
// 2N = 8192 the two column passes hold 32 points per thread instead (256 threads per row,
// radix 32 x 16 x 16: two exchanges and barriers instead of three; measured per 4096^2/50M
// apply, forward cols 4.28 -> 3.81 ms and inverse cols + fold 7.56 -> 6.90 ms, while the row
// passes, which also evaluate Z_p per point, were slower so: 5.32 -> 5.55 and 4.30 -> 4.61 ms).  The
// zero padding and the crop are exploited where they cost nothing: forward passes never
// load the zero half of their input (those points enter the first butterflies as
// constants), inverse passes store only the kept half of their output, and the
// column passes touch only the grid rows and tiles the bin's footprints reach.
#include <cstring>
#include <cstdio>

#include <map>
#include <mutex>

#include "internal.h"

namespace rimo {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
    float2 a0 = cadd(x0, x2), a1 = csub(x0, x2), a2 = cadd(x1, x3), a3 = mul_mi<INV>(csub(x1, x3));
    x0 = cadd(a0, a2);
    x2 = csub(a0, a2);
    x1 = cadd(a1, a3);
    x3 = csub(a1, a3);
}

#define RS2 0.70710678118654752440f
#define C16 0.92387953251128675613f
#define S16 0.38268343236508977173f

// W_N^k for the small radices: forward e^{-2 pi i k / N}, inverse its conjugate
template <bool INV>
__device__ __forceinline__ float2 w8(int k) {
    const float c[4] = {1.f, RS2, 0.f, -RS2};
    const float s[4] = {0.f, RS2, 1.f, RS2};
    return make_float2(c[k], INV ? s[k] : -s[k]);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    float2 o1 = cmul(v[3], w8<INV>(1)), o2 = cmul(v[5], w8<INV>(2)), o3 = cmul(v[7], w8<INV>(3));
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

template <bool INV>
__device__ __forceinline__ float2 w16(int k) {  // k in [0, 9]
    const float c[10] = {1.f, C16, RS2, S16, 0.f, -S16, -RS2, -C16, -1.f, -C16};
    const float s[10] = {0.f, S16, RS2, C16, 1.f, C16, RS2, S16, 0.f, -S16};
    return make_float2(c[k], INV ? s[k] : -s[k]);
}

// 16-point DFT as 4 x 4: inner DFT_4 over n1 (stride 4), twiddle W16^{n2 k1}, outer DFT_4.
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    // now v[n2 + 4 k1] = A[n2][k1]
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) v[n2 + 4 * k1] = cmul(v[n2 + 4 * k1], w16<INV>(n2 * k1));
    float2 t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 a = v[0 + 4 * k1], b = v[1 + 4 * k1], c = v[2 + 4 * k1], d = v[3 + 4 * k1];
        dft4<INV>(a, b, c, d);
        t[k1 + 0] = a;
        t[k1 + 4] = b;
        t[k1 + 8] = c;
        t[k1 + 12] = d;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = t[k];
}

// dft16 of an input whose points 4 .. 11 are zero (the first stage of a forward pass, whose
// row holds its samples in the centred half): the first layer of 4-point DFTs reduces to
// sums and differences of x_n2 and x_n2+12 (written out, since the compiler may not drop an
// addition of +0, which would turn -0 into +0)
template <bool INV>
__device__ __forceinline__ void dft16_hz(float2* v) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        const float2 a = v[n2], d = v[n2 + 12];
        const float2 md = mul_mi<INV>(make_float2(-d.x, -d.y));
        v[n2] = cadd(a, d);
        v[n2 + 8] = csub(a, d);
        v[n2 + 4] = cadd(a, md);
        v[n2 + 12] = csub(a, md);
    }
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) v[n2 + 4 * k1] = cmul(v[n2 + 4 * k1], w16<INV>(n2 * k1));
    float2 t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 a = v[0 + 4 * k1], b = v[1 + 4 * k1], c = v[2 + 4 * k1], d = v[3 + 4 * k1];
        dft4<INV>(a, b, c, d);
        t[k1 + 0] = a;
        t[k1 + 4] = b;
        t[k1 + 8] = c;
        t[k1 + 12] = d;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = t[k];
}

template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2* v) {
    if constexpr (R == 2) dft2<INV>(v[0], v[1]);
    else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 8) dft8<INV>(v);
    else dft16<INV>(v);
}

__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// One Stockham stage of radix R after NS points have been combined (NS * R <= N).
// Thread t owns butterflies j = t + q T (q < 16/R, T = N/16); butterfly j reads
// a[j + r N/R] and writes a'[(j / NS) NS R + j % NS + r NS].  Its twiddles
// W_{NS R}^{r (j mod NS)} come from the stage table tws[r NS + j mod NS], laid out so that
// consecutive threads read consecutive entries.
// HZ: a first stage whose inputs m = 4 .. 11 are zero (forward passes)
template <int N, int R, int NS, bool INV, bool FIRST, bool LAST, bool HZ = false>
__device__ __forceinline__ void fft_stage(float2 (&v)[16], float2* sm, int t, const float2* __restrict__ tws) {
    constexpr int T = N / 16;
    constexpr int Q = 16 / R;
    if (!FIRST) {
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) v[q * R + r] = sm[pidx(t + q * T + r * (N / R))];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (NS > 1) {
            const int jm = (t + q * T) & (NS - 1);
            if constexpr (R == 16) {
                // W^r for r = 1 .. 15 from two table entries (W and W^4), at most three
                // products deep: two loads instead of fifteen (fifteen loads from the table
                // were slower: 49.0 against 48.4 ms per 4096^2/50M apply)
                float2 w[16];
                w[1] = __ldg(&tws[NS + jm]);
                w[4] = __ldg(&tws[4 * NS + jm]);
                w[2] = cmul(w[1], w[1]);
                w[3] = cmul(w[2], w[1]);
                w[8] = cmul(w[4], w[4]);
#pragma unroll
                for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
#pragma unroll
                for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
#pragma unroll
                for (int r = 1; r < 16; ++r) v[q * R + r] = INV ? cmulc(v[q * R + r], w[r]) : cmul(v[q * R + r], w[r]);
            } else {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = __ldg(&tws[r * NS + jm]);
                    v[q * R + r] = INV ? cmulc(v[q * R + r], w) : cmul(v[q * R + r], w);
                }
            }
        }
        if constexpr (HZ && R == 16) dft16_hz<INV>(&v[q * R]);
        else dft_r<R, INV>(&v[q * R]);
    }
    if (!LAST) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int j = t + q * T;
            const int base = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
            for (int r = 0; r < R; ++r) sm[pidx(base + r * NS)] = v[q * R + r];
        }
        __syncthreads();
    }
}

// Radix plan of an L-point transform: 16, then 16s, then the remainder; L <= 256: two
// stages (16, L/16), L <= 4096: three (16, 16, L/256), L = 8192: four (16, 16, 16, 2).
// ----------------------------------------------------------------------------- 32 points per thread
// The 8192-point transform with 256 threads of 32 points (radix 32, 16, 16): two
// shared-memory exchanges instead of three.  Exchange buffer index i + i / 32 (the stride-32
// writes of the first stage spread over the banks).
__device__ __forceinline__ int pidx32(int i) { return i + (i >> 5); }

#define C32_1 0.98078528040323044913f
#define S32_1 0.19509032201612826785f
#define C32_3 0.83146961230254523708f
#define S32_3 0.55557023301960222474f

// W_32^k, k in [0, 16): forward e^{-2 pi i k / 32}, inverse its conjugate
template <bool INV>
__device__ __forceinline__ float2 w32(int k) {
    const float c[16] = {1.f, C32_1, C16, C32_3, RS2, S32_3, S16, S32_1, 0.f, -S32_1, -S16, -S32_3, -RS2, -C32_3, -C16, -C32_1};
    const float s[16] = {0.f, S32_1, S16, S32_3, RS2, C32_3, C16, C32_1, 1.f, C32_1, C16, C32_3, RS2, S32_3, S16, S32_1};
    return make_float2(c[k], INV ? s[k] : -s[k]);
}

// 32-point DFT in place: v[r] in natural order in and out (even / odd halves by dft16, then
// one radix-2 layer with W_32^k).  HZ: inputs 8 .. 23 are zero.
template <bool INV, bool HZ>
__device__ __forceinline__ void dft32(float2* v) {
    float2 e[16], o[16];
#pragma unroll
    for (int n = 0; n < 16; ++n) {
        e[n] = v[2 * n];
        o[n] = v[2 * n + 1];
    }
    if constexpr (HZ) {
        // e[n] = x[2n], o[n] = x[2n + 1]: zero for 2n (+1) in [8, 24), i.e. n in [4, 12)
        dft16_hz<INV>(e);
        dft16_hz<INV>(o);
    } else {
        dft16<INV>(e);
        dft16<INV>(o);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float2 t = k == 0 ? o[0] : cmul(o[k], w32<INV>(k));
        v[k] = cadd(e[k], t);
        v[k + 16] = csub(e[k], t);
    }
}

// tws32 layout as in DevTables.  In: v[m] = element t + 256 m.  Out: v[s] is element
// out_k32(t, s).  All 256 threads of the row must call it.
template <bool INV, bool HZ>
__device__ __forceinline__ void fft8192_32(float2 (&v)[32], float2* sm, int t, const float2* __restrict__ tw) {
    dft32<INV, HZ>(v);  // stage 1: butterfly j = t, outputs at 32 t + r
#pragma unroll
    for (int r = 0; r < 32; ++r) sm[pidx32(32 * t + r)] = v[r];
    __syncthreads();
    // stage 2: NS = 32, R = 16, butterflies j = t + 256 q, reads j + 512 r
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 16; ++r) v[16 * q + r] = sm[pidx32(t + 256 * q + 512 * r)];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = t + 256 * q, jm = j & 31;
        float2 w[16];
        w[1] = __ldg(&tw[32 + jm]);
        w[4] = __ldg(&tw[4 * 32 + jm]);
        w[2] = cmul(w[1], w[1]);
        w[3] = cmul(w[2], w[1]);
        w[8] = cmul(w[4], w[4]);
#pragma unroll
        for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
#pragma unroll
        for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
#pragma unroll
        for (int r = 1; r < 16; ++r) v[16 * q + r] = INV ? cmulc(v[16 * q + r], w[r]) : cmul(v[16 * q + r], w[r]);
        dft16<INV>(&v[16 * q]);
        const int base = (j >> 5) * 512 + jm;
#pragma unroll
        for (int r = 0; r < 16; ++r) sm[pidx32(base + 32 * r)] = v[16 * q + r];
    }
    __syncthreads();
    // stage 3: NS = 512, R = 16, butterflies j = t + 256 q (< 512), reads j + 512 r
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 16; ++r) v[16 * q + r] = sm[pidx32(t + 256 * q + 512 * r)];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int jm = t + 256 * q;
        const float2* __restrict__ tw3 = tw + 512;
        float2 w[16];
        w[1] = __ldg(&tw3[512 + jm]);
        w[4] = __ldg(&tw3[4 * 512 + jm]);
        w[2] = cmul(w[1], w[1]);
        w[3] = cmul(w[2], w[1]);
        w[8] = cmul(w[4], w[4]);
#pragma unroll
        for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
#pragma unroll
        for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
#pragma unroll
        for (int r = 1; r < 16; ++r) v[16 * q + r] = INV ? cmulc(v[16 * q + r], w[r]) : cmul(v[16 * q + r], w[r]);
        dft16<INV>(&v[16 * q]);
    }
}
// output index of v[s] after fft8192_32 in thread t: j = t + 256 (s / 16), k = j + 512 (s mod 16)
__device__ __forceinline__ int out_k32(int t, int s) { return t + 256 * (s >> 4) + 512 * (s & 15); }

template <int N>
struct Plan16 {
    static constexpr int STAGES = N <= 256 ? 2 : (N <= 4096 ? 3 : 4);
    static constexpr int R_LAST = N <= 256 ? N / 16 : (N <= 4096 ? N / 256 : N / 4096);
};

// In: v[m] = element t + T m of the input.  Out: element t + T m of the output is
// v[out_slot<N>(m)].  All threads of the block must call it (block-wide barriers).
// tws: the stage twiddle tables of length N (see stage_twiddles on the host): the second
// stage's W_{16 R}^{r j} at [0, 16 R), the third stage's W_{256 R}^{r j} at [256, 256 + 256 R),
// a fourth stage's W_{4096 R}^{r j} at [4352, 4352 + 4096 R).
template <int N, bool INV, bool HZ = false>
__device__ __forceinline__ void fft_n(float2 (&v)[16], float2* sm, int t, const float2* __restrict__ tws) {
    constexpr int RL = Plan16<N>::R_LAST;
    if constexpr (Plan16<N>::STAGES == 2) {
        fft_stage<N, 16, 1, INV, true, false, HZ>(v, sm, t, tws);
        fft_stage<N, RL, 16, INV, false, true>(v, sm, t, tws);
    } else if constexpr (Plan16<N>::STAGES == 3) {
        fft_stage<N, 16, 1, INV, true, false, HZ>(v, sm, t, tws);
        fft_stage<N, 16, 16, INV, false, false>(v, sm, t, tws);
        fft_stage<N, RL, 256, INV, false, true>(v, sm, t, tws + 256);
    } else {
        fft_stage<N, 16, 1, INV, true, false, HZ>(v, sm, t, tws);
        fft_stage<N, 16, 16, INV, false, false>(v, sm, t, tws);
        fft_stage<N, 16, 256, INV, false, false>(v, sm, t, tws + 256);
        fft_stage<N, RL, 4096, INV, false, true>(v, sm, t, tws + 256 + 4096);
    }
}

template <int N>
__device__ __forceinline__ int out_slot(int m) {
    constexpr int RL = Plan16<N>::R_LAST;
    constexpr int Q = 16 / RL;
    return (m % Q) * RL + m / Q;
}

// e^{-2 pi i w dn} from the double-float phase w * dn, reduced modulo 1 before sincos.
// The product and reduction keep ~48 significant bits (error-free FMA product), which is
// the FP64-accurate w-phase argument; only the final sincospi is single precision.
__device__ __forceinline__ float2 wphase(float w_hi, float w_lo, float2 d) {
    float p = w_hi * d.x;
    float e = fmaf(w_hi, d.x, -p);
    e = fmaf(w_hi, d.y, e);
    e = fmaf(w_lo, d.x, e);
    float k = rintf(p);
    float r = (p - k) + e;
    float s, c;
    sincospif(2.0f * r, &s, &c);
    return make_float2(c, -s);
}

struct ZArgs {
    const float4* zq;   // quarter table [|i_c|][|j_c|]: (n - 1) as a float pair, |Z_p|
    int zq_ld;
    float w_hi, w_lo;
};

// Z_p(i, j) = gc_x gc_y [/ n] e^{-2 pi i w (n - 1)} at (l_j, m_i): one table load (the grid
// correction and the w-term depend on |i_c|, |j_c| only)
__device__ __forceinline__ float2 z_factor(const ZArgs& z, int i, int j, int ic, int jc) {
    (void)i;
    (void)j;
    const float4 q = __ldg(&z.zq[abs(ic) * z.zq_ld + abs(jc)]);
    const float2 ph = wphase(z.w_hi, z.w_lo, make_float2(q.x, q.y));
    return make_float2(ph.x * q.z, ph.y * q.z);
}

// ----------------------------------------------------------------------------- bound
// Bound on the grid-step contributions of Phi^dagger Phi x.  Every forward-grid value of
// every w-bin is a sum of Z_p x over the pixels with unit-modulus twiddles, and the
// w-phase has unit modulus, so |X| <= B_x = sum_l (|x_l.re| + |x_l.im|) |Z_l|; a
// de-gridded y_k then has |y_k.x| + |y_k.y| <= sqrt(2) T1 B_x (T1 = max tap sum), and a
// contribution component at most tmax times that.  2 tmax T1 B_x goes to
// d_fx[FX_MAXTERM].  Per-block partial sums are added by the last block in block order
// (the bound, hence the scales, do not depend on timing).  Non-finite x sets status 3.
__global__ void __launch_bounds__(256) image_bound_kernel(const float2* __restrict__ x, int nx, int ny, ZArgs z,
                                                          uint32_t* fx, int* status) {
    __shared__ float red[256];
    __shared__ bool last;
    float acc = 0.f;
    bool bad = false;
    const int n = nx * ny;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int i = e / nx, j = e - i * nx;
        const float g = __ldg(&z.zq[abs(i - ny / 2) * z.zq_ld + abs(j - nx / 2)]).z;  // |Z_p|
        const float2 v = x[e];
        const float m = fabsf(v.x) + fabsf(v.y);
        bad |= !(m <= 3.4028234e38f);
        acc = fmaf(m, fabsf(g), acc);
    }
    if (bad) atomicExch(status, 3);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        reinterpret_cast<float*>(fx + FX_PART)[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(fx + FX_COUNT, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    float t = 0.f;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(reinterpret_cast<const float*>(fx + FX_PART) + b);
    red[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float mt = 2.f * __uint_as_float(__ldcg(fx + FX_TMAX)) * __uint_as_float(__ldcg(fx + FX_T1)) * red[0];
        if (!(mt <= 3.4028234e38f)) atomicExch(status, 3);
        fx[FX_MAXTERM] = __float_as_uint(mt);
        fx[FX_BX] = __float_as_uint(red[0]);
        fx[FX_COUNT] = 0u;
    }
}

// ----------------------------------------------------------------------------- clusters
// Transposed stores are made cluster-wide: the C CTAs of a thread-block cluster hold C x RB
// consecutive rows (or columns) in their shared memory; after a cluster barrier each CTA
// writes 1/C of the outputs for all C x RB of them, reading its partners' rows through
// distributed shared memory, so that every global write is C x RB x 8 contiguous bytes
// (32 bytes, one whole sector, for C x RB = 4) instead of RB x 8.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// a barrier that orders no memory: all its arrivals' remote reads have returned already
__device__ __forceinline__ void cluster_sync_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t dsmem_map(const void* ptr, uint32_t rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(ptr);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 dsmem_ld2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}

// The oversampled transforms: one L = 2N point transform per row (16 values per thread,
// T = L/16 = N/8 threads).  Forward: the centred N samples (c = j - N/2 in [-N/2, N/2)) sit
// at positions c mod L of the zero-padded input, i.e. thread slots m < 4 (c = t + T m) and
// m >= 12 (c = t + T m - L); the other slots are zero.  Inverse: of the L outputs only
// c mod L with c in [-N/2, N/2) (the crop) are kept.

// Transposed store of a CTA's (C = 1) or a cluster's (C > 1) rows: output row dst(kk) of
// `out` (leading dimension ld) gets, at columns [r0, r0 + C RB), value src(kk) of each of
// the C RB rows, for the nk kept values kk with keep(kk) (the others are not written).  With C > 1, after a cluster barrier each CTA
// writes nk / C of them for all the cluster's rows, reading partners' rows through
// distributed shared memory (32-byte writes for C RB = 4).
template <int RB, int C, int SR, int NK, int THREADS, class Src, class Dst, class Keep>
__device__ __forceinline__ void transposed_store(float2* smem, Src src, Dst dst, Keep keep, float2* out, size_t ld,
                                                 int r0_block) {  // r0_block: this CTA's first row
    if constexpr (C == 1) {
        __syncthreads();
        constexpr int NP = RB / 2;
        for (int e = threadIdx.x; e < NK * NP; e += THREADS) {
            const int kk = e / NP, q = e % NP;
            if (!keep(kk)) continue;
            const int k = src(kk);
            const float2 a = smem[(2 * q) * SR + pidx(k)], b = smem[(2 * q + 1) * SR + pidx(k)];
            *reinterpret_cast<float4*>(&out[(size_t)dst(kk) * ld + r0_block + 2 * q]) = make_float4(a.x, a.y, b.x, b.y);
        }
        __syncthreads();
    } else {
        cluster_sync_all();
        constexpr int NP = C * RB / 2, KPC = NK / C;
        static_assert(THREADS % NP == 0, "a thread keeps one row pair");
        const int rank = (int)(blockIdx.x % C);
        const int rbase = r0_block - rank * RB;  // first row of the cluster
        const int q = threadIdx.x % NP;                   // rows 2q, 2q + 1 of the cluster
        const uint32_t b0 = dsmem_map(smem + ((2 * q) % RB) * SR, (2 * q) / RB);
        const uint32_t b1 = dsmem_map(smem + ((2 * q + 1) % RB) * SR, (2 * q + 1) / RB);
        for (int e = threadIdx.x; e < KPC * NP; e += THREADS) {
            const int kk = rank * KPC + e / NP;
            if (!keep(kk)) continue;
            const uint32_t off = (uint32_t)pidx(src(kk)) * 8u;
            const float2 a = dsmem_ld2(b0 + off), b = dsmem_ld2(b1 + off);
            *reinterpret_cast<float4*>(&out[(size_t)dst(kk) * ld + rbase + 2 * q]) = make_float4(a.x, a.y, b.x, b.y);
        }
        cluster_sync_relaxed();  // partners are done reading before the block may exit
    }
}

// ----------------------------------------------------------------------------- row selection
// The column passes transform only the grid rows u of uv-tile rows holding a needed tile
// (tiles no footprint of the bin reaches are neither stored nor read): block b takes rows
// [row[b / bpt] * RG bpt + (b % bpt) RG, + RG), bpt = TS / RG blocks per tile row.  A
// cluster's blocks stay within one tile row (bpt is a multiple of C).  With on = 0 block b
// takes rows [b RG, + RG).  `bits` marks the selected tile rows for the last pass.
struct RowSel {
    int on, bpt, shift;
    uint32_t bits[8];
    uint16_t row[256];
};

__device__ __forceinline__ int sel_row0(const RowSel& sel, int b, int rows_per_blk) {
    return sel.on ? ((int)sel.row[b / sel.bpt] * sel.bpt + b % sel.bpt) * rows_per_blk : b * rows_per_blk;
}

// ----------------------------------------------------------------------------- jobs
// A pass over one (plan, w-bin) is a job.  A launch covers one job (the applies of a plan,
// bin after bin: the job's arguments by value) or a table of jobs of the same transform
// shape (a wideband batch, every channel's every bin in one launch per pass): job j owns
// the launch's blocks [first[j], first[j + 1]), and a block finds its job by bisection and
// then runs as in a one-job launch, with its block index within the job.
struct RowsJob {          // a rows pass: image rows -> transposed half transforms, or back
    const float2* in;
    float2* out;
    ZArgs z;
    RowSel sel;
};
struct ColsJob {          // a cols pass over the selected grid rows
    const float2* in;
    float2* out;
    const uint8_t* need;  // [tu * ntv + tv] of the job's bin: the tile is read or stored
    RowSel sel;
};
template <class J>
struct JobTable {
    const J* jobs;
    const int* first;     // njobs + 1 block offsets (multiples of the cluster size)
    int njobs;
};

// This block's job and its block index b within the job.
template <bool TABLE, class J>
__device__ __forceinline__ const J& block_job(const J& one, const JobTable<J>& tab, int& b) {
    b = (int)blockIdx.x;
    if constexpr (TABLE) {
        const int j = job_of(tab.first, tab.njobs, b);
        b -= __ldg(tab.first + j);
        return tab.jobs[j];
    } else {
        (void)tab;
        return one;
    }
}

// ----------------------------------------------------------------------------- forward rows
// grid: ny / RB blocks of RB * N/8 threads per job; block b transforms image rows
// [b RB, b RB + RB): Z_p times the row, zero-padded to 2N, DFT along l; row i of the result
// is column i of At (At[k][i], k < 2N).
template <int N, int RB, int C, bool TABLE>
__global__ void __launch_bounds__(RB * N / 8, (1024 / (RB * N / 8)) > 0 ? (1024 / (RB * N / 8)) : 1)
    fwd_rows_kernel(const __grid_constant__ RowsJob one, const JobTable<RowsJob> tab, int ny,
                    const float2* __restrict__ tws) {
    constexpr int L = 2 * N, T = L / 16, SR = L + L / 16;
    extern __shared__ float2 smem[];
    int bk;
    const RowsJob& J = block_job<TABLE>(one, tab, bk);
    const float2* __restrict__ x = J.in;
    const ZArgs z = J.z;
    const RowSel& sel = J.sel;
    const int g = threadIdx.x / T, t = threadIdx.x % T;
    float2* sm = smem + g * SR;
    const int i = bk * RB + g;
    const int ic = i - ny / 2;
    const float2* xr = x + (size_t)i * N;
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (m >= 4 && m < 12) {
            v[m] = make_float2(0.f, 0.f);
        } else {
            const int p = t + T * m;
            const int jc = m < 4 ? p : p - L;
            const int j = jc + N / 2;
            v[m] = cmul(__ldg(&xr[j]), z_factor(z, i, j, ic, jc));
        }
    }
    fft_n<L, false, true>(v, sm, t, tws);
#pragma unroll
    for (int m = 0; m < 16; ++m) sm[pidx(t + T * m)] = v[out_slot<L>(m)];
    // rows k of At the forward column pass does not transform are not stored
    transposed_store<RB, C, SR, L, RB * N / 8>(
        smem, [](int kk) { return kk; }, [](int kk) { return kk; },
        [&](int kk) { return !sel.on || ((sel.bits[(kk >> sel.shift) >> 5] >> ((kk >> sel.shift) & 31)) & 1u); },
        J.out, (size_t)ny, bk * RB);
}

// ----------------------------------------------------------------------------- forward cols
// grid: the selected grid rows / RG blocks per job; row u of At (N = ny samples) ->
// X[u][0 .. 2N).  Tiles of X that no active patch reads are not stored.
template <int N, int RG, bool TABLE>
__global__ void __launch_bounds__(RG * N / 8, (1024 / (RG * N / 8)) > 0 ? (1024 / (RG * N / 8)) : 1)
    fwd_cols_kernel(const __grid_constant__ ColsJob one, const JobTable<ColsJob> tab, int shift,
                    const float2* __restrict__ tws) {
    constexpr int L = 2 * N, T = L / 16, SR = L + L / 16;
    extern __shared__ float2 smem[];
    int bk;
    const ColsJob& J = block_job<TABLE>(one, tab, bk);
    const uint8_t* __restrict__ need = J.need;
    const int ntv = L >> shift;
    uint8_t* s_need = reinterpret_cast<uint8_t*>(smem + RG * SR);
    const int g = threadIdx.x / T, t = threadIdx.x % T;
    float2* sm = smem + g * SR;
    const int r0 = sel_row0(J.sel, bk, RG);
    const size_t u = (size_t)r0 + g;
    const float2* __restrict__ in = J.in + u * N;
    float2* __restrict__ out = J.out + u * L;
    for (int e = threadIdx.x; e < RG * ntv; e += blockDim.x) {
        const size_t uu = (size_t)r0 + e / ntv;
        s_need[e] = need[(uu >> shift) * ntv + e % ntv];
    }
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (m >= 4 && m < 12) {
            v[m] = make_float2(0.f, 0.f);
        } else {
            const int p = t + T * m;
            const int jc = m < 4 ? p : p - L;
            v[m] = __ldg(&in[jc + N / 2]);
        }
    }
    __syncthreads();
    fft_n<L, false, true>(v, sm, t, tws);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int k = t + T * m;
        if (s_need[g * ntv + (k >> shift)]) out[k] = v[out_slot<L>(m)];
    }
}

// The same pass for N = 4096 with 256 threads of 32 points per row (one row per block).
template <bool TABLE>
__global__ void __launch_bounds__(256, 2)
    fwd_cols32_kernel(const __grid_constant__ ColsJob one, const JobTable<ColsJob> tab, int shift,
                      const float2* __restrict__ tw) {
    constexpr int N = 4096, L = 8192;
    extern __shared__ float2 smem[];
    int bk;
    const ColsJob& J = block_job<TABLE>(one, tab, bk);
    const uint8_t* __restrict__ need = J.need;
    const int ntv = L >> shift;
    uint8_t* s_need = reinterpret_cast<uint8_t*>(smem + L + L / 32);
    const int t = threadIdx.x;
    const int r0 = sel_row0(J.sel, bk, 1);
    const size_t u = (size_t)r0;
    const float2* __restrict__ in = J.in + u * N;
    float2* __restrict__ out = J.out + u * L;
    for (int e = threadIdx.x; e < ntv; e += blockDim.x) s_need[e] = need[(u >> shift) * ntv + e];
    float2 v[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        if (m >= 8 && m < 24) {
            v[m] = make_float2(0.f, 0.f);
        } else {
            const int p = t + 256 * m;
            const int jc = m < 8 ? p : p - L;
            v[m] = __ldg(&in[jc + N / 2]);
        }
    }
    __syncthreads();
    fft8192_32<false, true>(v, smem, t, tw);
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int k = out_k32(t, q);
        if (s_need[k >> shift]) out[k] = v[q];
    }
}

// Inverse cols, N = 4096, 256 threads of 32 points per row, 4-CTA clusters for the store.
template <bool TABLE>
__global__ void __launch_bounds__(256, 2)
    inv_cols32_kernel(const __grid_constant__ ColsJob one, const JobTable<ColsJob> tab, int gx, int shift,
                      const float2* __restrict__ tw) {
    constexpr int N = 4096, L = 8192, SR = L + L / 16;
    extern __shared__ float2 smem[];
    int bk;
    const ColsJob& J = block_job<TABLE>(one, tab, bk);
    const uint8_t* __restrict__ need = J.need;
    const int ntv = L >> shift;
    uint8_t* s_need = reinterpret_cast<uint8_t*>(smem + SR);
    const int t = threadIdx.x;
    const int r0 = sel_row0(J.sel, bk, 1);
    const int u = r0;
    for (int e = threadIdx.x; e < ntv; e += blockDim.x) s_need[e] = need[(size_t)(u >> shift) * ntv + e];
    __syncthreads();
    const float2* __restrict__ in = J.in + (size_t)u * L;
    float2 v[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const int p = t + 256 * m;
        v[m] = s_need[p >> shift] ? __ldg(&in[p]) : make_float2(0.f, 0.f);
    }
    fft8192_32<true, false>(v, smem, t, tw);
#pragma unroll
    for (int q = 0; q < 32; ++q) smem[pidx(out_k32(t, q))] = v[q];
    transposed_store<1, 4, SR, N, 256>(
        smem, [](int kk) { return kk < N / 2 ? kk : kk + N; },
        [](int kk) { return kk < N / 2 ? kk + N / 2 : kk - N / 2; }, [](int) { return true; }, J.out, (size_t)gx, r0);
}

// ----------------------------------------------------------------------------- patch fold
// The gridded grid Xh of one bin is the sum of the accumulator patches of its active
// uv-tiles: a cell gets its own tile's patch and the halos of the tiles before it along u
// and v.  One block folds one needed tile (TS x TS cells) and writes it to Xh; tiles no
// patch reaches are never written and read as zero by the inverse transform.
struct FoldArgs {
    const float2* patch;   // [slot][PW * PW]
    const int2* slotbox;   // [tu * ntv + tv] -> (slot or -1, the slot's box: cells outside it
                           //   are zero and not stored), or null: `slot` with whole patches
    const int* slot;       // [tu * ntv + tv] -> slot or -1 (this bin)
    const int* tiles;      // needed tiles of this bin, tu * ntv + tv
    float2* Xh;            // [gx][gy]
    int ntu, ntv, TS, H, PW, gy;
};

// TSC: the tile side (32 or 64) as a compile-time constant, so the cell indexing is shifts
template <bool TABLE, int TSC>
__global__ void __launch_bounds__(256) fold_kernel(const __grid_constant__ FoldArgs one, const JobTable<FoldArgs> tab) {
    int bk;
    const FoldArgs& F = block_job<TABLE>(one, tab, bk);
    constexpr int TS = TSC;
    const int tile = F.tiles[bk];
    const int tu = tile / F.ntv, tv = tile - tu * F.ntv;
    const int tu1 = tu == 0 ? F.ntu - 1 : tu - 1, tv1 = tv == 0 ? F.ntv - 1 : tv - 1;
    const size_t np = (size_t)F.PW * F.PW;
    const uint32_t whole = box_pack(0, F.PW, 0, F.PW);
    // slot and box of tile t (an empty box for a tile without a patch)
    auto get = [&](int t, int& sl) {
        if (F.slotbox) {
            const int2 q = F.slotbox[t];
            sl = q.x;
            return sl < 0 ? 0u : (uint32_t)q.y;
        }
        sl = F.slot[t];
        return sl < 0 ? 0u : whole;
    };
    int s00, s10, s01, s11;
    const uint32_t x00 = get(tu * F.ntv + tv, s00), x10 = get(tu1 * F.ntv + tv, s10);
    const uint32_t x01 = get(tu * F.ntv + tv1, s01), x11 = get(tu1 * F.ntv + tv1, s11);
    // a box in the tile's cells (a, b): patch cells (a + oa, b + ob) with (oa, ob) the tile's
    // offset in that patch; [lo, lo + n) per axis, compared unsigned (empty: n = 0)
    struct Rng {
        int a, na, b, nb;
    };
    auto rng = [&](uint32_t x, int oa, int ob) {
        Rng r;
        r.a = (int)(x & 255u) - oa;
        r.na = max(0, (int)((x >> 8) & 255u) - oa - r.a);
        r.b = (int)((x >> 16) & 255u) - ob;
        r.nb = max(0, (int)(x >> 24) - ob - r.b);
        return r;
    };
    auto in = [](const Rng& r, int a, int b) {
        return (unsigned)(a - r.a) < (unsigned)r.na && (unsigned)(b - r.b) < (unsigned)r.nb;
    };
    const Rng r00 = rng(x00, 0, 0), r10 = rng(x10, TS, 0), r01 = rng(x01, 0, TS), r11 = rng(x11, TS, TS);
    const float2* __restrict__ patch = F.patch;
    float2* __restrict__ Xh = F.Xh;
    // every box covers all the cells its patch gives this tile (dense units): no per-cell test
    auto covers = [](const Rng& r, int na, int nb) { return r.a <= 0 && r.a + r.na >= na && r.b <= 0 && r.b + r.nb >= nb; };
    const bool dense = (s00 < 0 || covers(r00, TS, TS)) && (s10 < 0 || covers(r10, F.H, TS)) &&
                       (s01 < 0 || covers(r01, TS, F.H)) && (s11 < 0 || covers(r11, F.H, F.H));
    // one cell of the tile: the four sources (predicated), summed in a fixed order
    auto cell = [&](int e, float2& v) {
        const int a = e / TS, b = e - a * TS;
        const bool k00 = dense ? s00 >= 0 : in(r00, a, b);
        const bool k10 = dense ? (a < F.H && s10 >= 0) : in(r10, a, b);
        const bool k01 = dense ? (b < F.H && s01 >= 0) : in(r01, a, b);
        const bool k11 = dense ? (a < F.H && b < F.H && s11 >= 0) : in(r11, a, b);
        const float2 z = make_float2(0.f, 0.f);
        const float2 p00 = k00 ? __ldg(&patch[s00 * np + a * F.PW + b]) : z;
        const float2 p10 = k10 ? __ldg(&patch[s10 * np + (a + TS) * F.PW + b]) : z;
        const float2 p01 = k01 ? __ldg(&patch[s01 * np + a * F.PW + b + TS]) : z;
        const float2 p11 = k11 ? __ldg(&patch[s11 * np + (a + TS) * F.PW + b + TS]) : z;
        v = k00 ? p00 : z;
        if (k10) v = cadd(v, p10);
        if (k01) v = cadd(v, p01);
        if (k11) v = cadd(v, p11);
    };
    auto dst = [&](int e) {
        const int a = e / TS, b = e - a * TS;
        return Xh + (size_t)(tu * TS + a) * F.gy + tv * TS + b;
    };
    if constexpr (TS == 32) {
        // the four cells of a thread: every load issued before the stores (per 4096^2/50M
        // apply, inverse cols + fold 6.91 -> 6.72 ms against one cell at a time with a
        // runtime tile side; the 16 cells of a 64-wide tile at once took 80 registers and
        // slowed the wideband batch, 102.5 -> 114.2 ms, so 64-wide tiles go one at a time)
        float2 acc[4];
#pragma unroll
        for (int it = 0; it < 4; ++it) cell(threadIdx.x + 256 * it, acc[it]);
#pragma unroll
        for (int it = 0; it < 4; ++it) *dst(threadIdx.x + 256 * it) = acc[it];
    } else {
        for (int e = threadIdx.x; e < TS * TS; e += 256) {
            float2 v;
            cell(e, v);
            *dst(e) = v;
        }
    }
}

// ----------------------------------------------------------------------------- inverse cols
// grid: the selected grid rows / RB blocks per job; rows u of Xh (2N cells along v; cells
// of tiles without a mark in need[] are zero and not read) -> B[i][u] for the N image rows i.
template <int N, int RB, int C, bool TABLE>
__global__ void __launch_bounds__(RB * N / 8, (1024 / (RB * N / 8)) > 0 ? (1024 / (RB * N / 8)) : 1)
    inv_cols_kernel(const __grid_constant__ ColsJob one, const JobTable<ColsJob> tab, int gx, int shift,
                    const float2* __restrict__ tws) {
    constexpr int L = 2 * N, T = L / 16, SR = L + L / 16;
    extern __shared__ float2 smem[];
    int bk;
    const ColsJob& J = block_job<TABLE>(one, tab, bk);
    const uint8_t* __restrict__ need = J.need;
    const int ntv = L >> shift;
    uint8_t* s_need = reinterpret_cast<uint8_t*>(smem + RB * SR);
    const int g = threadIdx.x / T, t = threadIdx.x % T;
    float2* sm = smem + g * SR;
    const int r0 = sel_row0(J.sel, bk, RB);
    const int u = r0 + g;
    for (int e = threadIdx.x; e < RB * ntv; e += blockDim.x) {
        const int uu = r0 + e / ntv;
        s_need[e] = need[(size_t)(uu >> shift) * ntv + e % ntv];
    }
    __syncthreads();
    const float2* __restrict__ in = J.in + (size_t)u * L;
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int p = t + T * m;
        v[m] = s_need[g * ntv + (p >> shift)] ? __ldg(&in[p]) : make_float2(0.f, 0.f);
    }
    fft_n<L, true>(v, sm, t, tws);
#pragma unroll
    for (int m = 0; m < 16; ++m) sm[pidx(t + T * m)] = v[out_slot<L>(m)];
    // kept output kk < N: k = kk (kk < N/2) or kk + N; image row i = (k < N/2 ? k : k - L) + N/2
    transposed_store<RB, C, SR, N, RB * N / 8>(
        smem, [](int kk) { return kk < N / 2 ? kk : kk + N; },
        [](int kk) { return kk < N / 2 ? kk + N / 2 : kk - N / 2; }, [](int) { return true; }, J.out, (size_t)gx,
        r0);
}

// ----------------------------------------------------------------------------- inverse rows
// grid: ny / RG blocks; row i of B (2N cells along u) -> out[i][0 .. N) * conj(Z_p).
// With a table the grid is groups x ny / RG blocks: group c (the w-bins of one channel of a
// batch, jobs [group[c], group[c + 1])) has its bins summed into its image by the same
// block, one bin after the other (Sigma_p of Eq. 7 without a race or a second pass).
template <int N, int RG, bool TABLE>
__global__ void __launch_bounds__(RG * N / 8, (1024 / (RG * N / 8)) > 0 ? (1024 / (RG * N / 8)) : 1)
    inv_rows_kernel(const __grid_constant__ RowsJob one, const JobTable<RowsJob> tab, const int* __restrict__ group,
                    int ny, int accumulate, int real_only, const float2* __restrict__ tws) {
    constexpr int L = 2 * N, T = L / 16, SR = L + L / 16;
    extern __shared__ float2 smem[];
    const int g = threadIdx.x / T, t = threadIdx.x % T;
    float2* sm = smem + g * SR;
    int bk = (int)blockIdx.x, j0 = 0, j1 = 1;
    if constexpr (TABLE) {
        const int per = ny / RG, c = bk / per;
        bk -= c * per;
        j0 = __ldg(group + c);
        j1 = __ldg(group + c + 1);
    }
    const int i = bk * RG + g;
    const int ic = i - ny / 2;
    for (int jj = j0; jj < j1; ++jj) {
        const RowsJob& J = TABLE ? tab.jobs[jj] : one;
        const RowSel& sel = J.sel;
        const ZArgs z = J.z;
        const float2* __restrict__ in = J.in + (size_t)i * L;
        float2* __restrict__ orow = J.out + (size_t)i * N;
        const int acc = accumulate || jj > j0;
        float2 v[16];
        // columns u of tile rows the inverse column pass skipped are zero (not stored)
        uint32_t keep = 0xffffu;
        if (sel.on) {
            keep = 0;
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const int tr = (t + T * m) >> sel.shift;
                keep |= ((sel.bits[tr >> 5] >> (tr & 31)) & 1u) << m;
            }
        }
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = (keep >> m) & 1u ? __ldg(&in[t + T * m]) : make_float2(0.f, 0.f);
        fft_n<L, true>(v, sm, t, tws);
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int k = t + T * m;
            if (k >= N / 2 && k < 3 * N / 2) continue;  // outside the crop
            const int jc = k < N / 2 ? k : k - L;
            const int j = jc + N / 2;
            float2 val = cmulc(v[out_slot<L>(m)], z_factor(z, i, j, ic, jc));
            if (acc) val = cadd(val, orow[j]);
            if (real_only) val.y = 0.f;
            orow[j] = val;
        }
        // the next bin's first stage rewrites the exchange buffer this one's last stage read
        if (jj + 1 < j1) __syncthreads();
    }
}

// ----------------------------------------------------------------------------- Z_p
// Z_p(i, j) of every pixel, as the row passes apply it (for checking the w-phase).
__global__ void __launch_bounds__(256) zlayer_kernel(ZArgs z, int nx, int ny, float2* __restrict__ out) {
    const int64_t n = (int64_t)nx * ny;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / nx), j = (int)(e - (int64_t)i * nx);
        out[e] = z_factor(z, i, j, i - ny / 2, j - nx / 2);
    }
}

// ----------------------------------------------------------------------------- launchers
static ZArgs zargs(const rimo_plan* p, int bin) {
    ZArgs z;
    z.zq = p->tab.zq;
    z.zq_ld = p->nx / 2 + 1;
    z.w_hi = p->bins[bin].w_hi;
    z.w_lo = p->bins[bin].w_lo;
    return z;
}

void launch_zlayer(const rimo_plan* p, int bin, float2* out, cudaStream_t s) {
    const int64_t n = (int64_t)p->nx * p->ny;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8 * (int64_t)p->n_sm);
    zlayer_kernel<<<blocks, 256, 0, s>>>(zargs(p, bin), p->nx, p->ny, out);
}

void launch_image_bound(const rimo_plan* p, const float2* x, cudaStream_t s) {
    const int64_t n = (int64_t)p->nx * p->ny;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, std::min<int64_t>(FX_NPART, 4 * (int64_t)p->n_sm));
    image_bound_kernel<<<blocks, 256, 0, s>>>(x, p->nx, p->ny, zargs(p, 0), p->d_fx, p->d_status);
}

// rows per block of the 2N-point passes: 512 threads (N / 8 per row), ~70 KB of shared memory
template <int N>
static constexpr int rows_per_block() { return 4096 / N; }
// CTAs per cluster of the transposed-store passes: 4 rows per cluster, so that every write
// is one whole 32-byte sector (measured at 2N = 8192, forward-rows plus inverse-cols time
// per 32-bin apply: 13.1 ms with 4-row clusters, 14.4 ms with 8-row clusters and 64-byte
// writes, about 14.2 ms with 2-row clusters and 16-byte writes)
template <int RB>
static constexpr int cluster_of() { return RB >= 4 ? 1 : 4 / RB; }

template <class... KArgs, class... Args>
static void launch_clustered(void (*kernel)(KArgs...), int grid, int block, size_t smem, int C, cudaStream_t s,
                             Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    RIMO_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
}

// Raises a kernel's dynamic shared-memory limit once per (device, kernel, size).
template <class K>
static void set_smem(K kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    int dev = 0;
    RIMO_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = done[{dev, reinterpret_cast<const void*>(kernel)}];
    if (have < bytes) {
        RIMO_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        have = bytes;
    }
}

#define RIMO_DISPATCH_N(N_, CALL)                                                      \
    switch (N_) {                                                                      \
        case 64: { constexpr int NN = 64; CALL; } break;                               \
        case 128: { constexpr int NN = 128; CALL; } break;                             \
        case 256: { constexpr int NN = 256; CALL; } break;                             \
        case 512: { constexpr int NN = 512; CALL; } break;                             \
        case 1024: { constexpr int NN = 1024; CALL; } break;                           \
        case 2048: { constexpr int NN = 2048; CALL; } break;                           \
        case 4096: { constexpr int NN = 4096; CALL; } break;                           \
        default: fail(RIMO_ERR_INVALID_ARG, "unsupported transform length");           \
    }

// Row selection of `bin` for blocks of rpb rows (off when a block would span tile rows)
static RowSel row_sel(const rimo_plan* p, int bin, int rpb) {
    RowSel r;
    std::memset(&r, 0, sizeof(r));
    const auto& tr = p->trows[bin];
    const int ntu = p->gx / p->TS;
    if (rpb > p->TS || ntu > 256) return r;
    r.on = 1;
    r.bpt = p->TS / rpb;
    r.shift = p->TS == 64 ? 6 : 5;
    for (size_t i = 0; i < tr.size(); ++i) {
        r.row[i] = tr[i];
        r.bits[tr[i] >> 5] |= 1u << (tr[i] & 31);
    }
    return r;
}
static int sel_blocks(const rimo_plan* p, int bin, const RowSel& r, int rpb) {
    return r.on ? (int)p->trows[bin].size() * r.bpt : p->gx / rpb;
}
// the forward column pass's selection (blocks of 4096 / ny rows), shared with the forward
// row pass that writes its input
static RowSel fwd_sel(const rimo_plan* p, int bin) { return row_sel(p, bin, 4096 / p->ny); }
// the inverse column pass's selection (blocks of RB rows, clusters of C blocks; transform
// length 2 ny), shared with the inverse row pass that reads its output
static RowSel inv_sel(const rimo_plan* p, int bin) {
    const int RB = 4096 / p->ny, C = RB >= 4 ? 1 : 4 / RB;
    return row_sel(p, bin, C * RB <= p->TS ? RB : p->TS + 1);
}

static RowsJob rows_job(const rimo_plan* p, int bin, const float2* in, float2* out, const RowSel& sel) {
    RowsJob J;
    std::memset(&J, 0, sizeof(J));
    J.in = in;
    J.out = out;
    J.z = zargs(p, bin);
    J.sel = sel;
    return J;
}
static ColsJob cols_job(const rimo_plan* p, int bin, const float2* in, float2* out, const RowSel& sel) {
    ColsJob J;
    std::memset(&J, 0, sizeof(J));
    J.in = in;
    J.out = out;
    J.need = p->d_need + (size_t)bin * (size_t)(p->gx / p->TS) * (p->gy / p->TS);
    J.sel = sel;
    return J;
}
// grid-step patches (one per active tile, merged) or holographic-apply patches (one per
// needed tile): both cover [tile origin, + PW) on each axis
// the grid step's patches (slots and boxes from the plan) or, with `hslot`, the holographic
// apply's whole patches
static FoldArgs fold_args(const rimo_plan* p, int bin, const float2* patch, const int* hslot, float2* Xh) {
    const int ntu = p->gx / p->TS, ntv = p->gy / p->TS;
    FoldArgs F;
    F.patch = patch;
    F.slotbox = hslot ? nullptr : p->d_slot + (size_t)bin * ntu * ntv;
    F.slot = hslot ? hslot + (size_t)bin * ntu * ntv : nullptr;
    F.tiles = p->d_need_list + p->bins[bin].n0;
    F.Xh = Xh;
    F.ntu = ntu;
    F.ntv = ntv;
    F.TS = p->TS;
    F.H = p->H;
    F.PW = p->PW;
    F.gy = p->gy;
    return F;
}
static int tile_shift(int TS) { return TS == 64 ? 6 : 5; }

// One launch of each pass, for one job (TABLE = false: `one`) or a job table.
template <int N, bool TABLE>
static void run_fwd_rows(const RowsJob& one, const JobTable<RowsJob>& tab, int grid, int ny, const float2* tws,
                         cudaStream_t s) {
    constexpr int RB = rows_per_block<N>();
    constexpr int C = cluster_of<RB>();
    const size_t sm = (size_t)RB * (2 * N + N / 8) * sizeof(float2);
    if (grid == 0) return;
    if constexpr (C > 1) {
        if (grid % C != 0) fail(RIMO_ERR_UNSUPPORTED, "image rows do not fill the transposed-store clusters");
        set_smem(fwd_rows_kernel<N, RB, C, TABLE>, sm);
        launch_clustered(fwd_rows_kernel<N, RB, C, TABLE>, grid, RB * N / 8, sm, C, s, one, tab, ny, tws);
    } else {
        set_smem(fwd_rows_kernel<N, RB, 1, TABLE>, sm);
        fwd_rows_kernel<N, RB, 1, TABLE><<<grid, RB * N / 8, sm, s>>>(one, tab, ny, tws);
    }
}

// The column passes at 2N = 8192 use the 32-points-per-thread transform (tw32: the plan's
// tws32), the others the 16-point one.
template <int N, bool TABLE>
static void run_fwd_cols(const ColsJob& one, const JobTable<ColsJob>& tab, int grid, int TS, const float2* tws,
                         cudaStream_t s, const float2* tw32) {
    if constexpr (N == 4096) {
        if (!tw32) fail(RIMO_ERR_STATE, "8192-point column transforms without their twiddle table");
        const size_t sm = (size_t)(8192 + 8192 / 32) * sizeof(float2) + 8192 / 32 + 16;
        if (grid == 0) return;
        set_smem(fwd_cols32_kernel<TABLE>, sm);
        fwd_cols32_kernel<TABLE><<<grid, 256, sm, s>>>(one, tab, tile_shift(TS), tw32);
    } else {
        constexpr int RG = rows_per_block<N>();
        const int ntv = (2 * N) / TS;
        const size_t sm = (size_t)RG * (2 * N + N / 8) * sizeof(float2) + (size_t)RG * ntv + 16;
        if (grid == 0) return;
        set_smem(fwd_cols_kernel<N, RG, TABLE>, sm);
        fwd_cols_kernel<N, RG, TABLE><<<grid, RG * N / 8, sm, s>>>(one, tab, tile_shift(TS), tws);
    }
}

template <bool TABLE>
static void run_fold(const FoldArgs& one, const JobTable<FoldArgs>& tab, int grid, int TS, cudaStream_t s) {
    if (grid == 0) return;
    if (TS == 32) fold_kernel<TABLE, 32><<<grid, 256, 0, s>>>(one, tab);
    else fold_kernel<TABLE, 64><<<grid, 256, 0, s>>>(one, tab);  // plans hold TS = 32 or 64
}

template <int N, bool TABLE>
static void run_inv_cols(const ColsJob& one, const JobTable<ColsJob>& tab, int grid, int gx, int TS,
                         const float2* tws, cudaStream_t s, const float2* tw32) {
    if constexpr (N == 4096) {
        if (!tw32) fail(RIMO_ERR_STATE, "8192-point column transforms without their twiddle table");
        const size_t sm = (size_t)(8192 + 8192 / 16) * sizeof(float2) + 8192 / 32 + 16;
        if (grid == 0) return;
        if (grid % 4 != 0) fail(RIMO_ERR_UNSUPPORTED, "grid rows do not fill the transposed-store clusters");
        set_smem(inv_cols32_kernel<TABLE>, sm);
        launch_clustered(inv_cols32_kernel<TABLE>, grid, 256, sm, 4, s, one, tab, gx, tile_shift(TS), tw32);
    } else {
        constexpr int RB = rows_per_block<N>();
        constexpr int C = cluster_of<RB>();
        const int ntv = (2 * N) / TS;
        const size_t sm = (size_t)RB * (2 * N + N / 8) * sizeof(float2) + (size_t)RB * ntv + 16;
        if (grid == 0) return;
        // C consecutive blocks of a cluster stay in one tile row: TS / RB is a multiple of C
        if constexpr (C > 1) {
            if (grid % C != 0) fail(RIMO_ERR_UNSUPPORTED, "grid rows do not fill the transposed-store clusters");
            set_smem(inv_cols_kernel<N, RB, C, TABLE>, sm);
            launch_clustered(inv_cols_kernel<N, RB, C, TABLE>, grid, RB * N / 8, sm, C, s, one, tab, gx,
                             tile_shift(TS), tws);
        } else {
            set_smem(inv_cols_kernel<N, RB, 1, TABLE>, sm);
            inv_cols_kernel<N, RB, 1, TABLE><<<grid, RB * N / 8, sm, s>>>(one, tab, gx, tile_shift(TS), tws);
        }
    }
}

template <int N, bool TABLE>
static void run_inv_rows(const RowsJob& one, const JobTable<RowsJob>& tab, const int* group, int grid, int ny, int acc,
                         int re, const float2* tws, cudaStream_t s) {
    constexpr int RG = rows_per_block<N>();
    const size_t sm = (size_t)RG * (2 * N + N / 8) * sizeof(float2);
    if (grid == 0) return;
    set_smem(inv_rows_kernel<N, RG, TABLE>, sm);
    inv_rows_kernel<N, RG, TABLE><<<grid, RG * N / 8, sm, s>>>(one, tab, group, ny, acc, re, tws);
}

template <class J>
static JobTable<J> no_table() {
    JobTable<J> t;
    t.jobs = nullptr;
    t.first = nullptr;
    t.njobs = 0;
    return t;
}

template <int N>
static void fwd_rows(const rimo_plan* p, int bin, const float2* x, float2* At, cudaStream_t s) {
    run_fwd_rows<N, false>(rows_job(p, bin, x, At, fwd_sel(p, bin)), no_table<RowsJob>(),
                           p->ny / rows_per_block<N>(), p->ny, p->tab.tws_x, s);
}

template <int N>
static void fwd_cols(const rimo_plan* p, int bin, const float2* At, float2* X, cudaStream_t s) {
    const RowSel sel = fwd_sel(p, bin);
    run_fwd_cols<N, false>(cols_job(p, bin, At, X, sel), no_table<ColsJob>(),
                           sel_blocks(p, bin, sel, rows_per_block<N>()), p->TS, p->tab.tws_y, s, p->tab.tws32);
}

template <int N>
static void inv_cols(const rimo_plan* p, int bin, bool holo, float2* B, cudaStream_t s) {
    const auto& br = p->bins[bin];
    run_fold<false>(fold_args(p, bin, holo ? p->d_hpatch : p->d_patch, holo ? p->d_hslot : nullptr, p->d_X),
                    no_table<FoldArgs>(), br.n1 - br.n0, p->TS, s);
    const RowSel sel = inv_sel(p, bin);
    run_inv_cols<N, false>(cols_job(p, bin, p->d_X, B, sel), no_table<ColsJob>(),
                           sel_blocks(p, bin, sel, rows_per_block<N>()), p->gx, p->TS, p->tab.tws_y, s, p->tab.tws32);
}

template <int N>
static void inv_rows(const rimo_plan* p, int bin, const float2* B, float2* out, int acc, int re,
                     cudaStream_t s) {
    run_inv_rows<N, false>(rows_job(p, bin, B, out, inv_sel(p, bin)), no_table<RowsJob>(), nullptr,
                           p->ny / rows_per_block<N>(), p->ny, acc, re, p->tab.tws_x, s);
}

// ----------------------------------------------------------------------------- job tables
// The transform passes of a stage-batched apply: one launch per pass over every job.
struct WideFft {
    int nx = 0, ny = 0, gx = 0, TS = 0, ngroups = 0;
    const float2* tws_x = nullptr;
    const float2* tws_y = nullptr;
    const float2* tws32 = nullptr;
    struct Pass {
        void* jobs = nullptr;
        int* first = nullptr;
        int njobs = 0, blocks = 0;
    };
    Pass rows_fwd, cols_fwd, fold, cols_inv, rows_inv;
    int* group = nullptr;  // rows_inv: jobs of channel c are [group[c], group[c + 1])
    std::vector<void*> owned;
    ~WideFft() {
        for (void* q : owned) cudaFree(q);
    }
};

template <class J>
static WideFft::Pass upload_pass(WideFft* w, const std::vector<J>& jobs, const std::vector<int>& first,
                                 cudaStream_t s) {
    WideFft::Pass ps;
    ps.njobs = (int)jobs.size();
    ps.blocks = first.empty() ? 0 : first.back();
    if (jobs.empty()) return ps;
    void* dj = nullptr;
    void* df = nullptr;
    RIMO_CUDA(cudaMalloc(&dj, jobs.size() * sizeof(J)));
    w->owned.push_back(dj);
    RIMO_CUDA(cudaMalloc(&df, first.size() * sizeof(int)));
    w->owned.push_back(df);
    RIMO_CUDA(cudaMemcpyAsync(dj, jobs.data(), jobs.size() * sizeof(J), cudaMemcpyHostToDevice, s));
    RIMO_CUDA(cudaMemcpyAsync(df, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    ps.jobs = dj;
    ps.first = (int*)df;
    return ps;
}

WideFft* wide_fft_create(const std::vector<WideJob>& jobs, const std::vector<const float2*>& x,
                         const std::vector<float2*>& out, cudaStream_t s) {
    if (jobs.empty()) fail(RIMO_ERR_INVALID_ARG, "no jobs");
    auto* w = new WideFft();
    try {
        const rimo_plan* p0 = jobs[0].p;
        w->nx = p0->nx;
        w->ny = p0->ny;
        w->gx = p0->gx;
        w->TS = p0->TS;
        w->tws_x = p0->tab.tws_x;
        w->tws_y = p0->tab.tws_y;
        w->tws32 = p0->tab.tws32;
        w->ngroups = (int)x.size();
        const int rb = 4096 / p0->nx;  // rows per block of every pass (nx = ny)
        std::vector<RowsJob> rf, ri;
        std::vector<ColsJob> cf, ci;
        std::vector<FoldArgs> fo;
        std::vector<int> frf{0}, fcf{0}, ffo{0}, fci{0}, grp(w->ngroups + 1, 0);
        for (const WideJob& j : jobs) {
            const rimo_plan* p = j.p;
            const RowSel fs = fwd_sel(p, j.bin), is = inv_sel(p, j.bin);
            rf.push_back(rows_job(p, j.bin, x[j.group], j.AB, fs));
            frf.push_back(frf.back() + p->ny / rb);
            cf.push_back(cols_job(p, j.bin, j.AB, j.X, fs));
            fcf.push_back(fcf.back() + sel_blocks(p, j.bin, fs, rb));
            fo.push_back(fold_args(p, j.bin, j.patch, nullptr, j.X));
            ffo.push_back(ffo.back() + (p->bins[j.bin].n1 - p->bins[j.bin].n0));
            ci.push_back(cols_job(p, j.bin, j.X, j.AB, is));
            fci.push_back(fci.back() + sel_blocks(p, j.bin, is, rb));
            ri.push_back(rows_job(p, j.bin, j.AB, out[j.group], is));
            grp[j.group + 1]++;
        }
        for (int c = 0; c < w->ngroups; ++c) grp[c + 1] += grp[c];
        w->rows_fwd = upload_pass(w, rf, frf, s);
        w->cols_fwd = upload_pass(w, cf, fcf, s);
        w->fold = upload_pass(w, fo, ffo, s);
        w->cols_inv = upload_pass(w, ci, fci, s);
        w->rows_inv = upload_pass(w, ri, std::vector<int>{0, w->ngroups * (p0->ny / rb)}, s);
        RIMO_CUDA(cudaMalloc(&w->group, grp.size() * sizeof(int)));
        w->owned.push_back(w->group);
        RIMO_CUDA(cudaMemcpyAsync(w->group, grp.data(), grp.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        RIMO_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
    } catch (...) {
        delete w;
        throw;
    }
    return w;
}

void wide_fft_destroy(WideFft* w) { delete w; }

template <class J>
static JobTable<J> table_of(const WideFft::Pass& ps) {
    JobTable<J> t;
    t.jobs = (const J*)ps.jobs;
    t.first = ps.first;
    t.njobs = ps.njobs;
    return t;
}

template <int N>
static void wide_fwd_n(const WideFft* w, cudaStream_t s) {
    RowsJob r1;
    ColsJob c1;
    std::memset(&r1, 0, sizeof(r1));
    std::memset(&c1, 0, sizeof(c1));
    run_fwd_rows<N, true>(r1, table_of<RowsJob>(w->rows_fwd), w->rows_fwd.blocks, w->ny, w->tws_x, s);
    run_fwd_cols<N, true>(c1, table_of<ColsJob>(w->cols_fwd), w->cols_fwd.blocks, w->TS, w->tws_y, s, w->tws32);
}

template <int N>
static void wide_inv_n(const WideFft* w, int real_only, cudaStream_t s) {
    RowsJob r1;
    ColsJob c1;
    FoldArgs f1;
    std::memset(&r1, 0, sizeof(r1));
    std::memset(&c1, 0, sizeof(c1));
    std::memset(&f1, 0, sizeof(f1));
    run_fold<true>(f1, table_of<FoldArgs>(w->fold), w->fold.blocks, w->TS, s);
    run_inv_cols<N, true>(c1, table_of<ColsJob>(w->cols_inv), w->cols_inv.blocks, w->gx, w->TS, w->tws_y, s,
                          w->tws32);
    run_inv_rows<N, true>(r1, table_of<RowsJob>(w->rows_inv), w->group, w->rows_inv.blocks, w->ny, 0, real_only,
                          w->tws_x, s);
}

void wide_fwd(const WideFft* w, cudaStream_t s) { RIMO_DISPATCH_N(w->nx, wide_fwd_n<NN>(w, s)); }
void wide_inv(const WideFft* w, int real_only, cudaStream_t s) {
    RIMO_DISPATCH_N(w->nx, wide_inv_n<NN>(w, real_only, s));
}

void launch_fwd_rows(const rimo_plan* p, int bin, const float2* x, float2* At, cudaStream_t s) {
    RIMO_DISPATCH_N(p->nx, fwd_rows<NN>(p, bin, x, At, s));
}
void launch_fwd_cols(const rimo_plan* p, int bin, const float2* At, float2* X, cudaStream_t s) {
    RIMO_DISPATCH_N(p->ny, fwd_cols<NN>(p, bin, At, X, s));
}
void launch_inv_cols(const rimo_plan* p, int bin, float2* B, cudaStream_t s) {
    RIMO_DISPATCH_N(p->ny, inv_cols<NN>(p, bin, false, B, s));
}
void launch_inv_cols_from(const rimo_plan* p, int bin, bool holographic, float2* B, cudaStream_t s) {
    RIMO_DISPATCH_N(p->ny, inv_cols<NN>(p, bin, holographic, B, s));
}
void launch_inv_rows(const rimo_plan* p, int bin, const float2* B, float2* out, int accumulate,
                     int real_only, cudaStream_t s) {
    RIMO_DISPATCH_N(p->nx, inv_rows<NN>(p, bin, B, out, accumulate, real_only, s));
}

}  // namespace rimo
