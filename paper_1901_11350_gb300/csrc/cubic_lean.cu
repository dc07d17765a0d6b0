// cubic_lean.cu -- the stochastic Heun passes (App. B, Heun scheme with the
// thermal field of the stochastic LLG equation) on the shell-symmetric
// 27-point stencil, FP32, for one lattice without the dipole term whose xy
// plane is cut into whole 32 x 8 column tiles (nx % 32 == 0, ny % 8 == 0).
//
// The plane streaming is that of cubic.cu: a CTA owns a 32 x 8 column tile
// and a run of planes, planes pass through a ring of shared-memory tiles with
// a one-cell halo (four, finished two planes per block barrier), and each
// thread carries one plane's summary
// (centre spin c, the part w it gives the planes above and below, the open
// field accumulator) in registers from plane to plane.  What differs is the
// per-spin instruction budget of the loop, which bounds these passes:
//   * every tile record is read as one 16-byte vector and summed as two
//     f32x2 halves (x, y | z, pad), so no load is split and every vector sum
//     is two packed instructions;
//   * whole tiles only: no per-spin ownership tests;
//   * the ring slot of every plane is a compile-time offset (the plane loop
//     is unrolled by the ring size), staging addresses are fixed per segment
//     and the halo slots that lie outside an open lattice are zeroed once
//     per segment;
//   * the thermal field is a template switch, and the multi-function-unit
//     operations (log2, reciprocal square root, sine, cosine) are the
//     flush-to-zero forms, which give the same values on the normal
//     arguments they receive here;
//   * the parts of Philox rounds 0 and 1 that do not depend on the site are
//     computed once per launch on the host (the same bits: 18 of the 20
//     32 x 32 -> 64 multiplications remain per site).
#include <type_traits>

#include "internal.h"
#include "cubic.h"

namespace spgb {

namespace {

constexpr int LX = 32, LY = 8, LT = LX * LY;       // column tile = threads per CTA
constexpr int LHX = LX + 2, LHN = LHX * (LY + 2);  // halo tile: 34 x 10 records
// planes finished between two block barriers (2, 3 or 4): a group of LK
// planes is one cp.async group, fetched one group ahead into a ring of 2 LK
// plane buffers (measured at 128^3: pairs 50.8 G spin-updates/s, three per
// barrier 50.4, four 49.9 (spills), one plane per barrier with a ring of
// three fetched two planes ahead 49.3)
#ifndef SPGB_LEAN_LK
#define SPGB_LEAN_LK 2
#endif
constexpr int LK = SPGB_LEAN_LK;
static_assert(LK >= 2 && LK <= 4, "2 to 4 planes per barrier");
constexpr int LNB = 2 * LK;  // plane ring
#ifndef SPGB_LEAN_MINB
#define SPGB_LEAN_MINB 4
#endif
// 1: the folded term q travels as its x in the pad word of the predicted
// record and (y, z) in an 8-byte record (the step moves the method's 80 B per
// spin instead of 96); 0: q as a 16-byte record of its own
#ifndef SPGB_LEAN_PACKQ
#define SPGB_LEAN_PACKQ 1
#endif
constexpr unsigned kQRec = SPGB_LEAN_PACKQ ? 8u : 16u;  // bytes of a q record in its array and ring
#ifndef SPGB_LEAN_MINB_CORR
#define SPGB_LEAN_MINB_CORR 3
#endif
// the same with two columns per thread
#ifndef SPGB_LEAN_MINB2
#define SPGB_LEAN_MINB2 2
#endif
#ifndef SPGB_LEAN_MINB2_CORR
#define SPGB_LEAN_MINB2_CORR 2
#endif

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16(unsigned s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp8(unsigned s, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ float2 lds2(unsigned s)
{
    float2 r;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(s));
    return r;
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void wait_groups() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void st_zero(unsigned s)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %1, %1, %1};\n" ::"r"(s), "f"(0.f) : "memory");
}

// multi-function-unit operations, flush-to-zero forms
__device__ __forceinline__ float lg2f(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqf(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sinf_(float x)
{
    float r;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float cosf_(float x)
{
    float r;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int V> using I_ = std::integral_constant<int, V>;
// f(I_<0>), f(I_<1>), .. f(I_<K-1>) in order
template <typename F, int... J> __device__ __forceinline__ void each(F &&f, std::integer_sequence<int, J...>)
{
    (f(I_<J>{}), ...);
}

// A record as two f32x2 halves: a = (x, y), b = (z, pad).  Tile records are
// loaded and summed in this form (one 16-byte load each); the pad lane is
// carried through those sums and never read back.
struct p4 {
    float2 a, b;
};
// the record at shared-memory byte address s + OFF.  The compiler picks one
// 16-byte or two 8-byte loads (forcing 16-byte loads by inline PTX was
// measured slower: the quad-register destinations cost spills)
template <int OFF> __device__ __forceinline__ p4 ld4(unsigned s)
{
    const float4 v = *reinterpret_cast<const float4 *>(__cvta_shared_to_generic((unsigned)((int)s + OFF)));
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ p4 operator+(p4 u, p4 v) { return {__fadd2_rn(u.a, v.a), __fadd2_rn(u.b, v.b)}; }
// u - v (v times -1 is exact, so one rounding, as a subtraction)
__device__ __forceinline__ p4 minus(p4 u, p4 v, float2 m1)
{
    return {__ffma2_rn(v.a, m1, u.a), __ffma2_rn(v.b, m1, u.b)};
}

// A 3-vector as (x, y) in one f32x2 register pair and z: the form of the
// values carried from plane to plane (no pad lane to keep live).
struct pv {
    float2 a;
    float z;
};
__device__ __forceinline__ pv pvof(p4 u) { return {u.a, u.b.x}; }
__device__ __forceinline__ pv operator+(pv u, pv v) { return {__fadd2_rn(u.a, v.a), u.z + v.z}; }
__device__ __forceinline__ pv pfma(float2 s, pv u, pv v) { return {__ffma2_rn(s, u.a, v.a), fmaf(s.x, u.z, v.z)}; }
__device__ __forceinline__ pv pmul(float2 s, pv u) { return {__fmul2_rn(s, u.a), s.x * u.z}; }
__device__ __forceinline__ v3<float> v3of(pv u) { return {u.a.x, u.a.y, u.z}; }

__device__ __forceinline__ v3<float> unit(v3<float> a) { return rsqf(dot(a, a)) * a; }

// A(n, B) of Eq. 3 for a field already in units of c = -gamma/((1+alpha^2) mu):
// B + alpha n x B (the kernels receive the stencil constants, the on-site
// terms and the noise amplitude multiplied by c, so the field they form is
// c B and no per-spin scaling is left)
__device__ __forceinline__ v3<float> lA(float al, v3<float> n, v3<float> B) { return axpy(al, cross(n, B), B); }

// Philox4x32-10 of the counter (i, step, replica 8) for the sites of one
// launch.  Only the site index i differs between threads: half of round 0
// (the product of the counter's third word) and half of round 1 (the product
// of round 0's first output word) are the same for every site and are
// computed once on the host; the rest is the published round function.
struct LeanRng {
    uint32_t wk;      // replica 8 ^ k1                 (round 0, third output word)
    uint32_t yk;      // lo(M1 step_hi) ^ k0'           (round 1, first output word)
    uint32_t hk;      // hi(M0 x1) ^ k1'                (round 1, third output word)
    uint32_t l1;      // lo(M0 x1)                      (round 1, fourth output word)
    uint32_t rk[16];  // round keys of rounds 2 .. 9
};
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
__device__ __forceinline__ uint4 lean_bits(const LeanRng &G, uint32_t i)
{
    const uint32_t z1 = __umulhi(kPhiloxM0, i) ^ G.wk, w1 = kPhiloxM0 * i;
    uint4 c = make_uint4(__umulhi(kPhiloxM1, z1) ^ G.yk, kPhiloxM1 * z1, w1 ^ G.hk, G.l1);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ G.rk[2 * r], lo1, hi0 ^ c.w ^ G.rk[2 * r + 1], lo0);
    }
    return c;
}
// the launch-uniform words of rounds 0 and 1 for the counter's step and
// replica (x1 = round 0's first output word)
LeanRng lean_rng(const LlgConst<float> &c)
{
    auto hi = [](uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); };
    const uint32_t slo = (uint32_t)c.step, shi = (uint32_t)(c.step >> 32);
    const uint32_t x1 = hi(kPhiloxM1, shi) ^ slo ^ c.rk[0], y1 = kPhiloxM1 * shi;
    LeanRng G;
    G.wk = (c.replica * 8u) ^ c.rk[1];
    G.yk = y1 ^ c.rk[2];
    G.hk = hi(kPhiloxM0, x1) ^ c.rk[3];
    G.l1 = kPhiloxM0 * x1;
    for (int k = 0; k < 16; ++k) G.rk[k] = c.rk[4 + k];
    return G;
}

// Three standard normals from one Philox block by Box-Muller, scaled by the
// noise amplitude s: (u0, u1) -> eta_x, eta_y and (u2, u3) -> eta_z with
// u = (x + 1/2) 2^-32; sin and cos of 2 pi u are taken as -sin and -cos of
// 2 pi (u - 1/2), whose argument lies in (-pi, pi).
__device__ __forceinline__ v3<float> thermal(uint4 x, float s)
{
    const float k = 2.3283064365386963e-10f, h = 0.5f * 2.3283064365386963e-10f;
    const float twopi = 6.283185307179586f, pi = 3.141592653589793f;
    const float m2ln2 = -1.3862943611198906f;  // -2 ln 2 (x2 of the FP32 ln 2: exact)
    float u0 = fmaf((float)x.x, k, h), u1 = fmaf((float)x.y, k, h);
    float u2 = fmaf((float)x.z, k, h), u3 = fmaf((float)x.w, k, h);
    float t0 = fmaxf(m2ln2 * lg2f(u0), 1e-30f), t1 = fmaxf(m2ln2 * lg2f(u2), 1e-30f);
    float r0 = -s * (t0 * rsqf(t0)), r1 = -s * (t1 * rsqf(t1));
    float a = fmaf(twopi, u1, -pi), b = fmaf(twopi, u3, -pi);
    return {r0 * cosf_(a), r0 * sinf_(a), r1 * cosf_(b)};
}

// Summary of one plane at a thread's column (see cubic.cu): centre c, the
// part w = J1 c + J2 f + J3 k it gives the planes above and below, and the
// part e = J1 f + J2 k + in-plane face DMI it gives itself (f, k: sums of the
// four in-plane face and corner neighbours).
struct Sum {
    pv c, w, e;
    float cw;  // the centre record's pad word
};

// the exchange constants of the three shells as f32x2 pairs, and -1 for
// the packed subtractions (a kernel parameter, read from the constant bank)
struct LeanConst {
    float2 J1, J2, J3, m1;
};

// The summary of one column from its centre record c, the sums f and k of
// its in-plane face and corner neighbours and the face differences
// dx = n(+x) - n(-x), dy = n(+y) - n(-y).
template <int DM>
__device__ __forceinline__ Sum summary(const CubicParams<float> &P, const LeanConst &L, p4 c4, p4 f4, p4 k4, p4 dx4,
                                       p4 dy4)
{
    const pv c = pvof(c4), f = pvof(f4), k = pvof(k4);
    Sum r;
    r.c = c;
    r.cw = c4.b.y;
    r.w = pfma(L.J1, c, pfma(L.J2, f, pmul(L.J3, k)));
    pv e = pfma(L.J1, f, pmul(L.J2, k));
    if (DM != 0) {
        const pv dx = pvof(dx4), dy = pvof(dy4);
        if (DM == 1) {
            // D [(n(+x) - n(-x)) x xhat + (n(+y) - n(-y)) x yhat]
            const float D = P.Dx[0];
            e.a.x = fmaf(-D, dy.z, e.a.x);
            e.a.y = fmaf(D, dx.z, e.a.y);
            e.z = fmaf(D, dy.a.x - dx.a.y, e.z);
        } else {
            v3<float> ee = v3of(e) + cross(v3of(dx), mk(P.Dx[0], P.Dx[1], P.Dx[2])) +
                           cross(v3of(dy), mk(P.Dy[0], P.Dy[1], P.Dy[2]));
            e = {make_float2(ee.x, ee.y), ee.z};
        }
    }
    r.e = e;
    return r;
}

// Summaries of a thread's R columns (rows 0 .. R-1 of its strip, adjacent in
// y) in the plane of ring slot SLOT.  t: shared-memory address of the row-0
// centre record in slot 0; HN: records per ring slot.  Rows r-1, r, r+1 of
// column r are read once for both columns, and the sums follow one
// association for either R, so both give the same bits:
//   f = (n(x-1) + n(x+1)) + (n(y+1) + n(y-1)),
//   k = (n(x-1,y-1) + n(x+1,y-1)) + (n(x-1,y+1) + n(x+1,y+1)).
template <int DM, int R, int SLOT, int HN>
__device__ __forceinline__ void summarise(const CubicParams<float> &P, const LeanConst &L, unsigned t, Sum (&s)[R])
{
    constexpr int B = SLOT * HN * 16, X = 16, Y = 16 * LHX;
    // row -1 (above row 0): its x-neighbour sum and centre
    p4 up_m = ld4<B - Y - X>(t), up_p = ld4<B - Y + X>(t);
    p4 up_s = up_m + up_p, up_c = ld4<B - Y>(t);
    p4 rm = ld4<B - X>(t), rp = ld4<B + X>(t);
    p4 r_s = rm + rp, r_c = ld4<B>(t), r_d = minus(rp, rm, L.m1);
    each([&](auto jj) {
        constexpr int J = decltype(jj)::value;
        // row J + 1 (below row J)
        const p4 dm = ld4<B + (J + 1) * Y - X>(t), dp = ld4<B + (J + 1) * Y + X>(t);
        const p4 d_s = dm + dp, d_c = ld4<B + (J + 1) * Y>(t);
        s[J] = summary<DM>(P, L, r_c, r_s + (d_c + up_c), up_s + d_s, r_d, minus(d_c, up_c, L.m1));
        up_s = r_s;
        up_c = r_c;
        r_s = d_s;
        r_c = d_c;
        r_d = minus(dp, dm, L.m1);
    }, std::make_integer_sequence<int, R>{});
}

// s * (c x D_{+z}) added to the (x, y, z) lanes of v
template <int DM> __device__ __forceinline__ pv add_zdmi(const CubicParams<float> &P, pv v, pv c, float s)
{
    if (DM == 1) {
        const float d = s * P.Dz[2];
        v.a.x = fmaf(d, c.a.y, v.a.x);
        v.a.y = fmaf(-d, c.a.x, v.a.y);
    } else if (DM == 2) {
        v3<float> z = cross(v3of(c), mk(P.Dz[0], P.Dz[1], P.Dz[2]));
        v.a.x = fmaf(s, z.x, v.a.x);
        v.a.y = fmaf(s, z.y, v.a.y);
        v.z = fmaf(s, z.z, v.z);
    }
    return v;
}

// on-site field mu B + 2 K (Khat . c) Khat added to v
__device__ __forceinline__ pv add_onsite(const CubicParams<float> &P, pv v, pv c)
{
    const float kn = 2.f * P.K * (P.Kh[0] * c.a.x + P.Kh[1] * c.a.y + P.Kh[2] * c.z);
    v.a.x += fmaf(kn, P.Kh[0], P.Bz[0]);
    v.a.y += fmaf(kn, P.Kh[1], P.Bz[1]);
    v.z += fmaf(kn, P.Kh[2], P.Bz[2]);
    return v;
}


// Halo tile of a 32 x 8R column tile: (32 + 2) x (8R + 2) records per ring
// slot, staged by the CTA's 256 threads, NSL records each at most.
template <int R> struct LTile {
    static constexpr int HN = LHX * (LY * R + 2);
    static constexpr int NSL = (HN + LT - 1) / LT;
};

// One segment: planes [za, zb) of the column tile at (x0, y0), each thread R
// columns adjacent in y.  PASS 0: the predictor on src = n (writes the
// predicted record with q's x in its pad word, and q's y, z); PASS 1: the
// corrector on src = np (q of each plane arrives with the ring, writes
// nout = n).  Plane p lives in ring slot (p - za + 1) % LNB; the LK planes
// a group fetches form one cp.async group, waited for at the start of the
// next group.
template <int PASS, int DM, bool TH, int R>
__device__ __forceinline__ void lean_segment(const CubicParams<float> &P, const LeanConst &L, const LlgConst<float> &c,
                                             const float4 *__restrict__ src, float4 *__restrict__ np,
                                             float4 *__restrict__ q, float4 *__restrict__ nout, const LeanRng &G,
                                             float4 *tiles, unsigned char *qt, int x0, int y0, int za, int zb)
{
    constexpr int HN = LTile<R>::HN, NSL = LTile<R>::NSL;
    const int tid = threadIdx.x, tx = tid & (LX - 1), ty = tid / LX;
    const int plane = P.nx * P.ny;  // N < 2^31
    // this thread stages halo records tid, tid + 256, .. of every plane:
    // their in-plane offsets (-1: outside an open lattice, -2: no such record)
    auto halo = [&](int e) {
        if (e >= HN) return -2;
        int gx = x0 - 1 + e % LHX, gy = y0 - 1 + e / LHX;
        bool in = true;
        if (P.per0)
            gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
        else
            in = gx >= 0 && gx < P.nx;
        if (P.per1)
            gy = gy < 0 ? gy + P.ny : (gy >= P.ny ? gy - P.ny : gy);
        else
            in = in && gy >= 0 && gy < P.ny;
        return in ? gy * P.nx + gx : -1;
    };
    int g[NSL];
#pragma unroll
    for (int k = 0; k < NSL; ++k) g[k] = halo(tid + k * LT);
    const unsigned sd = smem_addr(tiles + tid);
    const unsigned qd = smem_addr(qt + kQRec * tid);
    constexpr unsigned kSlot = 16u * HN, kQSlot = kQRec * LT * R;
    float2 *const q2 = reinterpret_cast<float2 *>(q);  // (y, z) of q, packed layout
#pragma unroll
    for (int b = 0; b < LNB; ++b)
#pragma unroll
        for (int k = 0; k < NSL; ++k)
            if (g[k] == -1) st_zero(sd + b * kSlot + k * 16u * LT);
    const int col = (y0 + R * ty) * P.nx + x0 + tx;  // row 0 of the thread's strip
    auto issue = [&](auto slot, int p) {
        constexpr unsigned S = decltype(slot)::value;
        if (p <= zb) {
            int pz = p;
            bool zin = true;
            if (P.per2) {
                pz += pz < 0 ? P.nz : 0;
                pz -= pz >= P.nz ? P.nz : 0;
            } else {
                zin = pz >= 0 && pz < P.nz;
            }
            if (zin) {
                const float4 *base = src + (size_t)pz * plane;
#pragma unroll
                for (int k = 0; k < NSL; ++k)
                    if (g[k] >= 0) cp16(sd + S * kSlot + k * 16u * LT, base + g[k]);
            } else {
#pragma unroll
                for (int k = 0; k < NSL; ++k)
                    if (g[k] != -2) st_zero(sd + S * kSlot + k * 16u * LT);
            }
            if (PASS == 1 && p - 1 >= za && p - 1 < zb) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const unsigned qs = qd + S * kQSlot + j * kQRec * LT;
                    const size_t qi = (size_t)(p - 1) * plane + col + j * P.nx;
                    if (SPGB_LEAN_PACKQ)
                        cp8(qs, q2 + qi);
                    else
                        cp16(qs, q + qi);
                }
            }
        }
    };
    // the thread's row-0 centre record in slot 0
    const unsigned tc = smem_addr(tiles + (R * ty + 1) * LHX + tx + 1);
    // planes za-1, za (slots 0, 1), then za+1 .. za+LK (slots 2 .. LK+1) in flight
    issue(I_<0>{}, za - 1);
    issue(I_<1>{}, za);
    commit();
    each([&](auto j) { issue(I_<2 + decltype(j)::value>{}, za + 1 + decltype(j)::value); },
         std::make_integer_sequence<int, LK>{});
    commit();
    wait_groups<1>();
    __syncthreads();
    pv acc[R], wcur[R], ccur[R];
    float qx[R];  // x of q of the plane being finished (packed layout, corrector)
    {
        Sum below[R], cur[R];
        summarise<DM, R, 0, HN>(P, L, tc, below);
        summarise<DM, R, 1, HN>(P, L, tc, cur);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            // the open accumulator of the plane being finished, its w and centre
            acc[j] = add_onsite(P, add_zdmi<DM>(P, cur[j].e + below[j].w, below[j].c, -1.f), cur[j].c);
            wcur[j] = cur[j].w;
            ccur[j] = cur[j].c;
            qx[j] = cur[j].cw;
        }
    }
    int i = za * plane + col;
    const float al = c.alpha, dt = c.dt, hdt = 0.5f * c.dt;
    // finish the next plane z, whose upper neighbour z+1 sits in ring slot
    // SN: B(z) = acc + w(z+1) + c(z+1) x D_{+z}; then plane z+1 opens
    // A(z+1) = e(z+1) + w(z) - c(z) x D_{+z} + onsite(c(z+1)).
    auto finish = [&](auto sn) {
        constexpr int SN = decltype(sn)::value;
        Sum up[R];
        summarise<DM, R, SN, HN>(P, L, tc, up);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int ij = i + j * P.nx;
            v3<float> qi;
            if (PASS == 1) {
                if (SPGB_LEAN_PACKQ) {
                    const float2 yz = lds2(qd + SN * kQSlot + j * kQRec * LT);
                    qi = mk(qx[j], yz.x, yz.y);
                } else {
                    qi = v3of(pvof(ld4<0>(qd + SN * kQSlot + j * kQRec * LT)));
                }
            }
            const pv Bp = add_zdmi<DM>(P, acc[j] + up[j].w, up[j].c, 1.f);
            acc[j] = add_onsite(P, add_zdmi<DM>(P, up[j].e + wcur[j], ccur[j], -1.f), up[j].c);
            const v3<float> n = v3of(ccur[j]), B = v3of(Bp);
            wcur[j] = up[j].w;
            ccur[j] = up[j].c;
            qx[j] = up[j].cw;
            if (PASS == 0) {
                v3<float> Bth = mk(0.f, 0.f, 0.f);
                if (TH) Bth = thermal(lean_bits(G, (uint32_t)ij), c.sig[0]);
                const v3<float> A = lA(al, n, B + Bth);
                const v3<float> f = cross(n, A);
                const v3<float> p = unit(axpy(dt, f, n));
                const v3<float> qv = TH ? axpy(hdt, f + cross(p, lA(al, p, Bth)), n) : axpy(hdt, f, n);
                if (SPGB_LEAN_PACKQ) {
                    np[ij] = make_float4(p.x, p.y, p.z, qv.x);
                    q2[ij] = make_float2(qv.y, qv.z);
                } else {
                    st(q, ij, qv);
                    st(np, ij, p);
                }
            } else {
                const v3<float> Ap = lA(al, n, B);
                st(nout, ij, unit(axpy(hdt, cross(n, Ap), qi)));
            }
        }
        i += plane;
    };
    // (a second copy of the loop for the segment's interior, without the
    // range tests of `issue`, was measured: it costs the predictor spills at
    // 64 registers and gains the corrector nothing at 80)
    // planes z .. z+LK-1: planes z+1 .. z+LK have landed in slots BASE ..
    // BASE+LK-1 (mod 2 LK); the other half of the ring, read before the
    // barrier, takes planes z+LK+1 .. z+2LK
    auto group = [&](auto base, int z) {
        constexpr int BASE = decltype(base)::value;
        wait_groups<0>();
        __syncthreads();
        each([&](auto j) { issue(I_<(BASE + LK + decltype(j)::value) % LNB>{}, z + LK + 1 + decltype(j)::value); },
             std::make_integer_sequence<int, LK>{});
        commit();
        each([&](auto j) {
            constexpr int J = decltype(j)::value;
            if (J == 0 || z + J < zb) finish(I_<(BASE + J) % LNB>{});
        }, std::make_integer_sequence<int, LK>{});
    };
    for (int z = za; z < zb; z += LNB) {
        group(I_<2>{}, z);
        if (z + LK >= zb) break;
        group(I_<2 + LK>{}, z + LK);
    }
    wait_groups<0>();
    __syncthreads();  // the next segment reuses the ring
}

// resident CTAs per SM each pass and column count is compiled for
template <int PASS, int R> struct LeanMinB {
    static constexpr int value = R == 1 ? (PASS == 0 ? SPGB_LEAN_MINB : SPGB_LEAN_MINB_CORR)
                                        : (PASS == 0 ? SPGB_LEAN_MINB2 : SPGB_LEAN_MINB2_CORR);
};

// Work: the (32 x 8R column tile, plane) units in tile-major order, CTA b
// takes units [b per, (b + 1) per) as runs of planes, one segment each.
template <int PASS, int DM, bool TH, int R>
__global__ void __launch_bounds__(LT, (LeanMinB<PASS, R>::value))
    k_lean(const __grid_constant__ CubicParams<float> P, const float4 *__restrict__ src, float4 *__restrict__ np,
           float4 *__restrict__ q, float4 *__restrict__ nout, const __grid_constant__ LlgConst<float> c,
           const __grid_constant__ LeanConst L, const __grid_constant__ LeanRng G, int per)
{
    __shared__ __align__(16) float4 tiles[LNB * LTile<R>::HN];
    __shared__ __align__(16) unsigned char qt[PASS == 1 ? LNB * LT * R * kQRec : 16];
    allow_dependents();
    wait_prerequisite();  // the previous pass wrote what this one reads
    // units: (tile, plane) pairs, fewer than 2^31 (N < 2^31 spins, 256 R per
    // tile and plane); one division per CTA, then the runs advance tile by tile
    const int tiles_x = P.nx / LX;
    const int total = tiles_x * (P.ny / (LY * R)) * P.nz;
    int u = blockIdx.x * per;
    const int u1 = min(u + per, total);
    if (u >= u1) return;
    const int tile = u / P.nz;
    int za = u - tile * P.nz;
    int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    while (u < u1) {
        const int zb = min(P.nz, za + (u1 - u));
        lean_segment<PASS, DM, TH, R>(P, L, c, src, np, q, nout, G, tiles, qt, tx * LX, ty * LY * R, za, zb);
        u += zb - za;
        za = 0;
        if (++tx == tiles_x) {
            tx = 0;
            ++ty;
        }
    }
}

template <int PASS, int DM, int R>
cudaError_t lean_launch(int grid, const CubicParams<float> &P, const float4 *src, float4 *np, float4 *q, float4 *nout,
                        const LlgConst<float> &c, int per, cudaStream_t st)
{
    const LeanConst L{make_float2(P.J1, P.J1), make_float2(P.J2, P.J2), make_float2(P.J3, P.J3),
                      make_float2(-1.f, -1.f)};
    const LeanRng G = lean_rng(c);
    if constexpr (PASS == 0)
        if (c.thermal)
            return launch_pdl(k_lean<PASS, DM, true, R>, dim3(grid), dim3(LT), 0, st, P, src, np, q, nout, c, L, G,
                              per);
    return launch_pdl(k_lean<PASS, DM, false, R>, dim3(grid), dim3(LT), 0, st, P, src, np, q, nout, c, L, G, per);
}

template <int PASS, int R>
cudaError_t lean_dm(int grid, const CubicParams<float> &P, const float4 *src, float4 *np, float4 *q, float4 *nout,
                    const LlgConst<float> &c, int per, cudaStream_t st)
{
    if (P.dmi_mode == 0) return lean_launch<PASS, 0, R>(grid, P, src, np, q, nout, c, per, st);
    if (P.dmi_mode == 1) return lean_launch<PASS, 1, R>(grid, P, src, np, q, nout, c, per, st);
    return lean_launch<PASS, 2, R>(grid, P, src, np, q, nout, c, per, st);
}

}  // namespace

bool cubic_lean_fits(int nx, int ny, int rows)
{
    return nx > 0 && ny > 0 && nx % LX == 0 && ny % (LY * (rows == 2 ? 2 : 1)) == 0;
}

cudaError_t launch_cubic_lean(int pass, const CubicParams<float> &P, const float4 *src, float4 *np, float4 *q,
                              float4 *nout, const LlgConst<float> &c, int per, cudaStream_t st, int rows)
{
    const int R = rows == 2 ? 2 : 1;
    const long total = (long)(P.nx / LX) * (P.ny / (LY * R)) * P.nz;
    if (total == 0) return cudaSuccess;
    if (per < 1) per = 1;
    const int grid = (int)((total + per - 1) / per);
    // every field term and the noise amplitude in units of c = cA[0] (one
    // atom per cell): the kernels form c B directly
    const float s = c.cA[0];
    CubicParams<float> Ps = P;
    Ps.J1 *= s;
    Ps.J2 *= s;
    Ps.J3 *= s;
    for (int k = 0; k < 3; ++k) {
        Ps.Dx[k] *= s;
        Ps.Dy[k] *= s;
        Ps.Dz[k] *= s;
        Ps.Bz[k] *= s;
    }
    Ps.K *= s;
    LlgConst<float> cs = c;
    cs.sig[0] *= s;
    if (R == 2)
        return pass == 0 ? lean_dm<0, 2>(grid, Ps, src, np, q, nout, cs, per, st)
                         : lean_dm<1, 2>(grid, Ps, src, np, q, nout, cs, per, st);
    return pass == 0 ? lean_dm<0, 1>(grid, Ps, src, np, q, nout, cs, per, st)
                     : lean_dm<1, 1>(grid, Ps, src, np, q, nout, cs, per, st);
}

int cubic_lean_resident_ctas(int pass, int rows)
{
    int n = 0;
    cudaError_t e;
    if (rows == 2)
        e = pass == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_lean<0, 1, true, 2>, LT, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_lean<1, 1, false, 2>, LT, 0);
    else
        e = pass == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_lean<0, 1, true, 1>, LT, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_lean<1, 1, false, 1>, LT, 0);
    return (e == cudaSuccess && n > 0) ? n : 1;
}

}  // namespace spgb
