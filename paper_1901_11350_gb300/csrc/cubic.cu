// cubic.cu -- the LLG predictor/corrector passes specialised to a one-atom
// lattice whose couplings live on the 3x3x3 cell neighbourhood with shell
// symmetry: exchange J1 on the 6 faces, J2 on the 12 edges, J3 on the 8
// corners, DMI vectors on the faces only (D_{-o} = -D_o).  This covers simple
// cubic lattices with up to three shells (bulk or interfacial DMI) and square
// lattices.
//
// Layout of the work: a CTA owns a TX x TY column tile of the xy plane and a
// chunk of ZC planes.  It streams planes z0-1 .. z0+ZC through a double
// buffer in shared memory ((TX+2) x (TY+2) records, halo included, filled
// with cp.async; periodic halos wrap, open ones are zero).  Each thread owns
// one column and keeps, for the last three planes, the centre spin c, the sum
// of its four in-plane face neighbours f and of its four in-plane corner
// neighbours k in registers, so that for the plane in the middle
//     shell 1 = f(z) + c(z-1) + c(z+1)
//     shell 2 = k(z) + f(z-1) + f(z+1)
//     shell 3 = k(z-1) + k(z+1)
// and the face DMI field is sum_axes (n(+o) - n(-o)) x D_o.  Every spin is read
// from global memory about (1 + 2/ZC)(1 + halo) times per pass (L2 serves the
// re-reads), and from shared memory 8 times.
#include <type_traits>

#include "internal.h"
#include "cubic.h"

namespace spgb {

namespace {

// resident CTAs per SM the register allocation is held to
#ifndef SPGB_CUBIC_MINB
#define SPGB_CUBIC_MINB 3
#endif
// resident CTAs per SM the corrector pass is compiled for (its own register
// budget: it has no thermal field to generate)
#ifndef SPGB_CUBIC_MINB_CORR
#define SPGB_CUBIC_MINB_CORR 4
#endif
// the same with two columns per thread (more state per thread)
#ifndef SPGB_CUBIC_MINB2
#define SPGB_CUBIC_MINB2 2
#endif
#ifndef SPGB_CUBIC_MINB2_CORR
#define SPGB_CUBIC_MINB2_CORR 2
#endif
// plane buffers in shared memory per pass (planes are fetched NB - 1 ahead)
// and how many planes ahead the corrector loads its folded term q (two
// planes ahead costs the 64-register corrector spills and time)
#ifndef SPGB_CUBIC_NB_PRED
#define SPGB_CUBIC_NB_PRED 3
#endif
#ifndef SPGB_CUBIC_NB_CORR
#define SPGB_CUBIC_NB_CORR 3
#endif
#ifndef SPGB_CUBIC_QAHEAD
#define SPGB_CUBIC_QAHEAD 1
#endif
// 1: the Heun corrector's folded term q travels with the plane ring (q of
// plane p - 1 in the cp.async group of plane p), read from shared memory;
// 0: loaded from global memory QAHEAD planes ahead into registers
#ifndef SPGB_CUBIC_QSMEM
#define SPGB_CUBIC_QSMEM 1
#endif
// 1: programmatic dependent launch of the passes (each waits for the one
// before it ahead of any global access; the launch overlaps its drain)
#ifndef SPGB_CUBIC_PDL
#define SPGB_CUBIC_PDL 1
#endif

// A CTA's 256 threads form TX x TY columns; each thread owns ROWS columns of
// the CTA's TX x (TY ROWS) tile, at rows ty, ty + TY, ..  (ROWS 1 or 2: the
// second column shares the thread's plane staging and loop work and gives it
// a second, independent stencil and thermal-field chain to interleave).
constexpr int TX = 32, TY = 8;
constexpr int HX = TX + 2;
template <int ROWS> struct Tile {
    static constexpr int TYE = TY * ROWS;                 // rows of the tile
    static constexpr int HN = HX * (TYE + 2);             // halo tile records
    static constexpr int NS = (HN + TX * TY - 1) / (TX * TY);  // halo records per thread
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ------------------------------------------------------------ arithmetic
// 3-vectors for the stencil sums: FP32 keeps (x, y) in a float2 so that the
// sums run on Blackwell's packed f32x2 pipe (one instruction per pair, the
// same IEEE rounding per component); FP64 uses plain v3<double>.
struct pv {
    float2 xy;
    float z;
};
__device__ __forceinline__ pv padd(pv a, pv b) { return {__fadd2_rn(a.xy, b.xy), a.z + b.z}; }
__device__ __forceinline__ pv psub(pv a, pv b) { return {__ffma2_rn(b.xy, make_float2(-1.f, -1.f), a.xy), a.z - b.z}; }
__device__ __forceinline__ pv paxpy(float s, pv a, pv b) { return {__ffma2_rn(make_float2(s, s), a.xy, b.xy), fmaf(s, a.z, b.z)}; }
__device__ __forceinline__ pv pscale(float s, pv a) { return {__fmul2_rn(make_float2(s, s), a.xy), s * a.z}; }
__device__ __forceinline__ v3<float> tov(pv a) { return {a.xy.x, a.xy.y, a.z}; }

template <typename T> __device__ __forceinline__ v3<T> padd(v3<T> a, v3<T> b) { return a + b; }
template <typename T> __device__ __forceinline__ v3<T> psub(v3<T> a, v3<T> b) { return a - b; }
template <typename T> __device__ __forceinline__ v3<T> paxpy(T s, v3<T> a, v3<T> b) { return axpy(s, a, b); }
template <typename T> __device__ __forceinline__ v3<T> pscale(T s, v3<T> a) { return s * a; }
template <typename T> __device__ __forceinline__ v3<T> tov(v3<T> a) { return a; }

// SPGB_SCALAR_STENCIL: plain scalar FP32 sums (for comparison with the packed form)
template <typename T> struct PV;
#ifdef SPGB_SCALAR_STENCIL
template <> struct PV<float> { using type = v3<float>; };
#else
template <> struct PV<float> { using type = pv; };
#endif
template <> struct PV<double> { using type = v3<double>; };
template <typename T> using pv_t = typename PV<T>::type;

template <typename P> __device__ __forceinline__ P tload_as(const float4 *t, int e);
template <> __device__ __forceinline__ pv tload_as<pv>(const float4 *t, int e)
{
    float4 v = t[e];
    return {make_float2(v.x, v.y), v.z};
}
template <> __device__ __forceinline__ v3<float> tload_as<v3<float>>(const float4 *t, int e) { return ldc(t, e); }
__device__ __forceinline__ pv_t<float> tload(const float4 *t, int e) { return tload_as<pv_t<float>>(t, e); }
__device__ __forceinline__ v3<double> tload(const dq4 *t, int e) { return ldc(t, e); }

// Box-Muller for FP32 from the multi-function unit: sin/cos of
// 2 pi (u - 1/2) in (-pi, pi) (so sin(2 pi u) = -sin, cos(2 pi u) = -cos), and
// sqrt(t) = t rsqrt(t).  Absolute error of eta ~1e-6.
__device__ __forceinline__ v3<float> box_muller_fast(uint4 x)
{
    const float s = 2.3283064365386963e-10f, h = 0.5f * 2.3283064365386963e-10f;
    const float twopi = 6.283185307179586f;
    float u0 = fmaf((float)x.x, s, h), u1 = fmaf((float)x.y, s, h);
    float u2 = fmaf((float)x.z, s, h), u3 = fmaf((float)x.w, s, h);
    float t0 = fmaxf(-2.f * __logf(u0), 1e-30f), t1 = fmaxf(-2.f * __logf(u2), 1e-30f);
    float r0 = t0 * rsqrtf(t0), r1 = t1 * rsqrtf(t1);
    float sa, ca;
    __sincosf(twopi * (u1 - 0.5f), &sa, &ca);
    float cb = __cosf(twopi * (u3 - 0.5f));
    return {-r0 * ca, -r0 * sa, -r1 * cb};
}
__device__ __forceinline__ v3<float> thermal_eta(uint4 x, float) { return box_muller_fast(x); }
__device__ __forceinline__ v3<double> thermal_eta(uint4 x, double) { return box_muller(x, 0.0); }

// ------------------------------------------------------------ plane staging
// The halo tile of a plane is (TX+2) x (TY+2) records; each thread copies at
// most two of them.  Their in-plane offsets (periodic wrap or "absent" for an
// open edge) do not depend on z and are computed once per CTA.
struct HaloSlot {
    int off;  // gy * nx + gx, or -1 outside the lattice in-plane
};

template <typename T, int ROWS>
__device__ __forceinline__ HaloSlot halo_slot(const CubicParams<T> &P, int x0, int y0, int e)
{
    HaloSlot h{-1};
    if (e >= Tile<ROWS>::HN) return h;
    int hx = e % HX, hy = e / HX;
    int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
    bool in = true;
    if (P.per0) {
        gx %= P.nx;
        gx += gx < 0 ? P.nx : 0;
    } else {
        in = in && gx >= 0 && gx < P.nx;
    }
    if (P.per1) {
        gy %= P.ny;
        gy += gy < 0 ? P.ny : 0;
    } else {
        in = in && gy >= 0 && gy < P.ny;
    }
    h.off = in ? gy * P.nx + gx : -1;
    return h;
}

template <typename T>
__device__ __forceinline__ void copy_rec(rec_t<T> *dst, const rec_t<T> *src)
{
    cp_async16(dst, src);
    if (sizeof(rec_t<T>) == 32) cp_async16(reinterpret_cast<char *>(dst) + 16, reinterpret_cast<const char *>(src) + 16);
}

template <typename T, int ROWS>
__device__ __forceinline__ void load_plane(const CubicParams<T> &P, const rec_t<T> *__restrict__ src, rec_t<T> *tile,
                                           const HaloSlot (&h)[Tile<ROWS>::NS], int z)
{
    bool zin = true;
    if (P.per2) {
        z += z < 0 ? P.nz : 0;
        z -= z >= P.nz ? P.nz : 0;
    } else {
        zin = z >= 0 && z < P.nz;
    }
    const rec_t<T> *plane = src + z * (P.nx * P.ny);
    rec_t<T> zero{};
#pragma unroll
    for (int k = 0; k < Tile<ROWS>::NS; ++k) {
        int e = threadIdx.x + k * TX * TY;
        if (k == 0 || e < Tile<ROWS>::HN) {
            if (zin && h[k].off >= 0)
                copy_rec<T>(tile + e, plane + h[k].off);
            else
                tile[e] = zero;
        }
    }
}

// Summary of one plane at a thread's column: its centre spin c, the part
// `w` it contributes to the planes above and below (exchange J1 c + J2 f +
// J3 k, f and k the sums of the four in-plane face and corner neighbours)
// and the part `e` it contributes to itself (J1 f + J2 k + in-plane face DMI).
template <typename T> struct Plane {
    v3<T> c, w, e;
};

// DM: 0 no DMI, 1 bulk (D_o = D ohat on the faces), 2 any face vectors
template <typename T, int DM>
__device__ __forceinline__ Plane<T> summarise(const CubicParams<T> &P, const rec_t<T> *tile, int tx, int ty)
{
    int e = (ty + 1) * HX + tx + 1;
    pv_t<T> c = tload(tile, e);
    pv_t<T> xp = tload(tile, e + 1), xm = tload(tile, e - 1);
    pv_t<T> yp = tload(tile, e + HX), ym = tload(tile, e - HX);
    pv_t<T> f = padd(padd(xp, xm), padd(yp, ym));
    pv_t<T> k = padd(padd(tload(tile, e + HX + 1), tload(tile, e - HX - 1)), padd(tload(tile, e - HX + 1), tload(tile, e + HX - 1)));
    Plane<T> r;
    r.c = tov(c);
    r.w = tov(paxpy(P.J1, c, paxpy(P.J2, f, pscale(P.J3, k))));
    v3<T> ee = tov(paxpy(P.J1, f, pscale(P.J2, k)));
    if (DM != 0) {
        v3<T> dx = tov(psub(xp, xm)), dy = tov(psub(yp, ym));
        if (DM == 1) {
            // D [(n(+x) - n(-x)) x xhat + (n(+y) - n(-y)) x yhat]
            T D = P.Dx[0];
            ee.x = fma(-D, dy.z, ee.x);
            ee.y = fma(D, dx.z, ee.y);
            ee.z = fma(D, dy.x - dx.y, ee.z);
        } else {
            ee = ee + cross(dx, mk(P.Dx[0], P.Dx[1], P.Dx[2])) + cross(dy, mk(P.Dy[0], P.Dy[1], P.Dy[2]));
        }
    }
    r.e = ee;
    return r;
}

// c x D_{+z}: the DMI field a spin c on the plane below gets from ... (sign
// applied by the caller)
template <typename T, int DM> __device__ __forceinline__ v3<T> zdmi(const CubicParams<T> &P, v3<T> c)
{
    if (DM == 0) return mk(T(0), T(0), T(0));
    if (DM == 1) return mk(P.Dz[2] * c.y, -P.Dz[2] * c.x, T(0));
    return cross(c, mk(P.Dz[0], P.Dz[1], P.Dz[2]));
}

// on-site part: Zeeman + anisotropy
template <typename T> __device__ __forceinline__ v3<T> onsite(const CubicParams<T> &P, v3<T> c)
{
    v3<T> Kh = mk(P.Kh[0], P.Kh[1], P.Kh[2]);
    T kn = T(2) * P.K * dot(Kh, c);
    return axpy(kn, Kh, mk(P.Bz[0], P.Bz[1], P.Bz[2]));
}

// One segment: planes [za, zb) of the column tile at (x0, y0).
//
// Streaming in z: when plane p+1 arrives the field of plane p is complete,
//     B(p) = A(p) + w(p+1) + c(p+1) x D_{+z},
// and plane p+1 opens its own accumulator
//     A(p+1) = e(p+1) + w(p) - c(p) x D_{+z} + onsite(c(p+1)),
// so only A, w and c of one plane stay live between iterations.
// PASS 0: predictor on n; PASS 1: corrector on np (q folded term, n out).
// Plane p lives in tiles[(p - za + 1) % NB]; every fetch is one cp.async
// group (empty past the segment's last plane), so that waiting for all but
// the newest NB - 2 groups means "the plane needed next has landed".
// REPL: the records belong to replica r of a batch (its noise amplitude and
// thermal stream); otherwise r is 0 and the amplitude is c.sig[0].
template <typename T, int SOLVER, int PASS, int DM, bool HAS_BDD, int NB, bool REPL, int ROWS>
__device__ __forceinline__ void segment(const CubicParams<T> &P, const rec_t<T> *__restrict__ src,
                                        rec_t<T> *__restrict__ np, rec_t<T> *__restrict__ q,
                                        rec_t<T> *__restrict__ nout, const rec_t<T> *__restrict__ Bdd,
                                        const LlgConst<T> &c, rec_t<T> (*tiles)[Tile<ROWS>::HN],
                                        rec_t<T> (*qt)[TX * TY * ROWS], int r, int x0, int y0, int za, int zb)
{
    constexpr bool QS = PASS == 1 && SOLVER == SP_HEUN && SPGB_CUBIC_QSMEM;
    static_assert(NB >= 2 && NB <= 4, "2 to 4 plane buffers");
    constexpr int QA = PASS == 1 && SOLVER != SP_RK4 ? SPGB_CUBIC_QAHEAD : 1;
    static_assert(QA >= 1 && QA <= 2, "q is fetched 1 or 2 planes ahead");
    constexpr int NS = Tile<ROWS>::NS;
    int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    int x = x0 + tx;
    bool own[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) own[j] = x < P.nx && y0 + ty + j * TY < P.ny;
    HaloSlot h[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) h[k] = halo_slot<T, ROWS>(P, x0, y0, threadIdx.x + k * TX * TY);
    const int plane_sz = P.nx * P.ny;  // N < 2^31
    // one cp.async group per ring slot: plane p of src (and, QS, q of plane
    // p - 1 at this thread's columns)
    auto load = [&](int slot, int p) {
        if (p <= zb) load_plane<T, ROWS>(P, src, tiles[slot], h, p);
#pragma unroll
        for (int j = 0; j < ROWS; ++j)
            if (QS && own[j] && p - 1 >= za && p - 1 < zb)
                copy_rec<T>(&qt[slot][threadIdx.x + j * TX * TY],
                            q + (size_t)(p - 1) * plane_sz + (y0 + ty + j * TY) * P.nx + x);
        cp_async_commit();
    };
    // planes za-1 .. za+NB-2 in flight
#pragma unroll
    for (int k = 0; k < NB; ++k) load(k, za - 1 + k);
    cp_async_wait<NB - 1>();
    __syncthreads();
    Plane<T> below[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) below[j] = summarise<T, DM>(P, tiles[0], tx, ty + j * TY);
    __syncthreads();
    load(0, za + NB - 1);
    cp_async_wait<NB - 1>();
    __syncthreads();
    v3<T> acc[ROWS], wcur[ROWS], ccur[ROWS];
    int i[ROWS];
    // per-spin global inputs of the planes being finished, fetched QA planes
    // (Bdd: one plane) ahead so that their latency overlaps the stencils
    v3<T> qa[ROWS][QA], bn[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        Plane<T> cur = summarise<T, DM>(P, tiles[1], tx, ty + j * TY);
        acc[j] = cur.e + below[j].w - zdmi<T, DM>(P, below[j].c) + onsite(P, cur.c);
        wcur[j] = cur.w;
        ccur[j] = cur.c;
        i[j] = za * plane_sz + (y0 + ty + j * TY) * P.nx + x;
        bn[j] = mk(T(0), T(0), T(0));
#pragma unroll
        for (int k = 0; k < QA; ++k) {
            qa[j][k] = mk(T(0), T(0), T(0));
            if (PASS == 1 && SOLVER != SP_RK4 && !QS && own[j] && za + k < zb) qa[j][k] = ld(q, i[j] + k * plane_sz);
        }
        if (HAS_BDD && own[j]) bn[j] = ld(Bdd, i[j]);
    }
    int s_next = 2 % NB, s_free = 1;  // slots of planes z+1 and z
    const uint64_t step = REPL && (PASS == 0 || SOLVER == SP_RK4) ? llg_step_of(c) : c.step;  // Philox step
    for (int z = za; z < zb; ++z) {
        const int sn = s_next, sf = s_free;  // plane z+1 (landed after the wait); plane z, summarised
        s_next = s_next + 1 == NB ? 0 : s_next + 1;
        s_free = s_free + 1 == NB ? 0 : s_free + 1;
        v3<T> qi[ROWS], bi[ROWS];
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            qi[j] = qa[j][0];
            bi[j] = bn[j];
#pragma unroll
            for (int k = 0; k + 1 < QA; ++k) qa[j][k] = qa[j][k + 1];
            if (own[j] && z + QA < zb && PASS == 1 && SOLVER != SP_RK4 && !QS)
                qa[j][QA - 1] = ld(q, i[j] + QA * plane_sz);
            if (HAS_BDD && own[j] && z + 1 < zb) bn[j] = ld(Bdd, i[j] + plane_sz);
        }
        cp_async_wait<NB - 2>();
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ROWS; ++j)
            if (QS && own[j]) qi[j] = ldc(qt[sn], threadIdx.x + j * TX * TY);  // q of plane z, landed with plane z+1
        load(sf, z + NB);
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            Plane<T> up = summarise<T, DM>(P, tiles[sn], tx, ty + j * TY);
            v3<T> B = acc[j] + up.w + zdmi<T, DM>(P, up.c);
            acc[j] = up.e + wcur[j] - zdmi<T, DM>(P, ccur[j]) + onsite(P, up.c);
            v3<T> ni = ccur[j];
            wcur[j] = up.w;
            ccur[j] = up.c;
            const int ii = i[j];
            i[j] += plane_sz;
            if (!own[j]) continue;
            if (HAS_BDD) B = B + bi[j];
            v3<T> Bth = mk(T(0), T(0), T(0));
            if ((PASS == 0 || SOLVER == SP_RK4) && c.thermal)
                Bth = (REPL ? c.rsig[r] : c.sig[0]) *
                      thermal_eta(REPL ? thermal_bits_at(c, step, (uint32_t)ii, (uint32_t)r)
                                       : thermal_bits_at(c, c.step, (uint32_t)ii, 0u),
                                  T(0));
            if (SOLVER == SP_RK4) {
                // stage PASS of the fourth-order Runge-Kutta step (the same
                // thermal field in every stage): np = next stage state, q =
                // accumulator k1 + 2 k2 + 2 k3, nout = n (read by stages 1-3,
                // written by stage 3)
                v3<T> k = cross(ni, llg_A(c.cA[0], c.alpha, ni, B + Bth));
                if (PASS == 0) {
                    st(q, ii, k);
                    st(np, ii, axpy(T(0.5) * c.dt, k, ni));
                } else {
                    v3<T> n0 = ldc(nout, ii);
                    if (PASS < 3) {
                        st(q, ii, axpy(T(2), k, ldc(q, ii)));
                        st(np, ii, axpy((PASS == 1 ? T(0.5) : T(1)) * c.dt, k, n0));
                    } else {
                        st(nout, ii, normalised(axpy(c.dt / T(6), ldc(q, ii) + k, n0)));
                    }
                }
            } else if (PASS == 0) {
                v3<T> A = llg_A(c.cA[0], c.alpha, ni, B + Bth);
                if (SOLVER == SP_HEUN) {
                    v3<T> f = cross(ni, A);
                    v3<T> p = normalised(axpy(c.dt, f, ni));
                    v3<T> g = cross(p, llg_A(c.cA[0], c.alpha, p, Bth));
                    st(np, ii, p);
                    st(q, ii, axpy(T(0.5) * c.dt, f + g, ni));
                } else if (SOLVER == SP_SIB) {
                    // np holds the midpoint (n + x_p)/2, q the thermal part of A there
                    v3<T> m = T(0.5) * (ni + sib_solve(ni, A, c.dt));
                    st(np, ii, m);
                    st(q, ii, llg_A(c.cA[0], c.alpha, m, Bth));
                } else {
                    v3<T> p = rotate(ni, A, c.dt);
                    st(np, ii, p);
                    st(q, ii, T(0.5) * (A + llg_A(c.cA[0], c.alpha, p, Bth)));
                }
            } else {
                v3<T> Ap = llg_A(c.cA[0], c.alpha, ni, B);
                if (SOLVER == SP_HEUN) {
                    st(nout, ii, normalised(axpy(T(0.5) * c.dt, cross(ni, Ap), qi[j])));
                } else if (SOLVER == SP_SIB) {
                    st(nout, ii, sib_solve(ldc(nout, ii), Ap + qi[j], c.dt));
                } else {
                    st(nout, ii, rotate(ldc(nout, ii), axpy(T(0.5), Ap, qi[j]), c.dt));
                }
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();  // the next segment reuses the tiles
}

// The work is the list of (column tile, plane) units, tile-major (and
// replica-major before that in a batch of replicas).  CTA b
// takes units [b*per, (b+1)*per): a few contiguous runs of planes, each
// streamed as one segment.  With per = units / (SMs x resident CTAs) every SM
// gets the same amount of work in a single wave.
// resident CTAs per SM a kernel's register allocation is held to
template <int SOLVER, int PASS, int ROWS> struct MinBlocks {
    static constexpr int value = ROWS == 1 ? (PASS == 0 || SOLVER == SP_RK4 ? SPGB_CUBIC_MINB : SPGB_CUBIC_MINB_CORR)
                                           : (PASS == 0 || SOLVER == SP_RK4 ? SPGB_CUBIC_MINB2 : SPGB_CUBIC_MINB2_CORR);
};

template <typename T, int SOLVER, int PASS, int DM, bool HAS_BDD, bool REPL, int ROWS>
__global__ void __launch_bounds__(TX *TY, (MinBlocks<SOLVER, PASS, ROWS>::value)) k_cubic(const __grid_constant__ CubicParams<T> P, const rec_t<T> *__restrict__ src,
                                                  rec_t<T> *__restrict__ np, rec_t<T> *__restrict__ q,
                                                  rec_t<T> *__restrict__ nout, const rec_t<T> *__restrict__ Bdd,
                                                  const LlgConst<T> c, int per)
{
    constexpr int NB = PASS == 0 || SOLVER == SP_RK4 ? SPGB_CUBIC_NB_PRED : SPGB_CUBIC_NB_CORR;
    constexpr bool QS = PASS == 1 && SOLVER == SP_HEUN && SPGB_CUBIC_QSMEM;
    __shared__ __align__(32) rec_t<T> tiles[NB][Tile<ROWS>::HN];
    __shared__ __align__(32) rec_t<T> qtiles[QS ? NB : 1][QS ? TX * TY * ROWS : 1];
    allow_dependents();
    wait_prerequisite();  // the previous pass reads what this one overwrites
    int tiles_x = (P.nx + TX - 1) / TX, tiles_y = (P.ny + Tile<ROWS>::TYE - 1) / Tile<ROWS>::TYE;
    long ntile = (long)tiles_x * tiles_y;
    long total = ntile * P.nz * (REPL ? llg_reps(c) : 1);
    long u = (long)blockIdx.x * per, u1 = min(u + per, total);
    while (u < u1) {
        long tg = u / P.nz;  // tile over all replicas
        int za = (int)(u % P.nz);
        int zb = (int)min((long)P.nz, za + (u1 - u));
        int r = REPL ? (int)(tg / ntile) : 0;
        int tile = (int)(tg - (long)r * ntile);
        size_t o = REPL ? (size_t)r * ((size_t)P.nx * P.ny * P.nz) : 0;
        segment<T, SOLVER, PASS, DM, HAS_BDD, NB, REPL, ROWS>(P, src + o, np ? np + o : np, q + o,
                                                              nout ? nout + o : nout, Bdd, c, tiles,
                                                              (rec_t<T>(*)[TX * TY * ROWS])qtiles, r,
                                                              (tile % tiles_x) * TX, (tile / tiles_x) * Tile<ROWS>::TYE,
                                                              za, zb);
        u += zb - za;
    }
}

template <typename K, typename T>
cudaError_t launch_one(K kern, int grid, const CubicParams<T> &P, const rec_t<T> *src, rec_t<T> *np, rec_t<T> *q,
                       rec_t<T> *nout, const rec_t<T> *Bdd, const LlgConst<T> &c, int per, cudaStream_t st)
{
#if SPGB_CUBIC_PDL
    return launch_pdl(kern, dim3(grid), dim3(TX * TY), 0, st, P, src, np, q, nout, Bdd, c, per);
#else
    kern<<<grid, TX * TY, 0, st>>>(P, src, np, q, nout, Bdd, c, per);
    return cudaGetLastError();
#endif
}

template <typename T, int DM, bool HB, bool RP, int RW>
cudaError_t launch_dmb(int pass, int solver, int grid, const CubicParams<T> &P, const rec_t<T> *src, rec_t<T> *np,
                       rec_t<T> *q, rec_t<T> *nout, const rec_t<T> *Bdd, const LlgConst<T> &c, int per,
                       cudaStream_t st)
{
    if (solver == SP_RK4) {  // stages 0..3, without the dipole term
        if constexpr (HB) {
            return cudaErrorNotSupported;
        } else {
            switch (pass) {
            case 0: return launch_one(k_cubic<T, SP_RK4, 0, DM, HB, RP, RW>, grid, P, src, np, q, nout, Bdd, c, per, st);
            case 1: return launch_one(k_cubic<T, SP_RK4, 1, DM, HB, RP, RW>, grid, P, src, np, q, nout, Bdd, c, per, st);
            case 2: return launch_one(k_cubic<T, SP_RK4, 2, DM, HB, RP, RW>, grid, P, src, np, q, nout, Bdd, c, per, st);
            default: return launch_one(k_cubic<T, SP_RK4, 3, DM, HB, RP, RW>, grid, P, src, np, q, nout, Bdd, c, per, st);
            }
        }
    }
    if (pass == 0) {
        if (solver == SP_HEUN)
            return launch_one(k_cubic<T, SP_HEUN, 0, DM, HB, RP, RW>, grid, P, src, np, q, nout, Bdd, c, per, st);
        if (solver == SP_SIB)
            return launch_one(k_cubic<T, SP_SIB, 0, DM, HB, RP, RW>, grid, P, src, np, q, nout, Bdd, c, per, st);
        return launch_one(k_cubic<T, SP_DEPONDT, 0, DM, HB, RP, RW>, grid, P, src, np, q, nout, Bdd, c, per, st);
    }
    if (solver == SP_HEUN)
        return launch_one(k_cubic<T, SP_HEUN, 1, DM, HB, RP, RW>, grid, P, src, np, q, nout, Bdd, c, per, st);
    if (solver == SP_SIB)
        return launch_one(k_cubic<T, SP_SIB, 1, DM, HB, RP, RW>, grid, P, src, np, q, nout, Bdd, c, per, st);
    return launch_one(k_cubic<T, SP_DEPONDT, 1, DM, HB, RP, RW>, grid, P, src, np, q, nout, Bdd, c, per, st);
}

// (a batch of replicas never carries the dipole field)
// (two columns per thread only for FP32 single lattices without the dipole
// field; other calls take one)
template <typename T, int DM>
cudaError_t launch_dm(int pass, int solver, int grid, const CubicParams<T> &P, const rec_t<T> *src, rec_t<T> *np,
                      rec_t<T> *q, rec_t<T> *nout, const rec_t<T> *Bdd, const LlgConst<T> &c, int per, int rows,
                      cudaStream_t st)
{
    if (llg_reps(c) > 1)
        return launch_dmb<T, DM, false, true, 1>(pass, solver, grid, P, src, np, q, nout, nullptr, c, per, st);
    if (Bdd) return launch_dmb<T, DM, true, false, 1>(pass, solver, grid, P, src, np, q, nout, Bdd, c, per, st);
    if constexpr (std::is_same<T, float>::value)
        if (rows == 2) return launch_dmb<T, DM, false, false, 2>(pass, solver, grid, P, src, np, q, nout, Bdd, c, per, st);
    return launch_dmb<T, DM, false, false, 1>(pass, solver, grid, P, src, np, q, nout, Bdd, c, per, st);
}

}  // namespace

template <typename T>
cudaError_t launch_cubic(int pass, int solver, const CubicParams<T> &P, const rec_t<T> *src, rec_t<T> *np, rec_t<T> *q,
                         rec_t<T> *nout, const rec_t<T> *Bdd, const LlgConst<T> &c, int per, cudaStream_t st, int rows,
                         bool lean)
{
    rows = cubic_rows_taken(sizeof(T) == 8 ? SP_F64 : SP_F32, rows, llg_reps(c) > 1, Bdd != nullptr);
    if constexpr (std::is_same<T, float>::value)
        if (lean && solver == SP_HEUN && pass <= 1 && !Bdd && llg_reps(c) == 1 && cubic_lean_fits(P.nx, P.ny, rows))
            return launch_cubic_lean(pass, P, src, np, q, nout, c, per, st, rows);
    long total = cubic_units(P.nx, P.ny, P.nz, rows) * llg_reps(c);
    if (total == 0) return cudaSuccess;
    if (per < 1) per = 1;
    int grid = (int)((total + per - 1) / per);
    if (P.dmi_mode == 0) return launch_dm<T, 0>(pass, solver, grid, P, src, np, q, nout, Bdd, c, per, rows, st);
    if (P.dmi_mode == 1) return launch_dm<T, 1>(pass, solver, grid, P, src, np, q, nout, Bdd, c, per, rows, st);
    return launch_dm<T, 2>(pass, solver, grid, P, src, np, q, nout, Bdd, c, per, rows, st);
}

int cubic_rows_taken(int prec, int rows, bool replicas, bool dipole)
{
    return (rows == 2 && prec == SP_F32 && !replicas && !dipole) ? 2 : 1;
}

long cubic_units(int nx, int ny, int nz, int rows)
{
    const int tye = TY * (rows == 2 ? 2 : 1);
    return (long)((nx + TX - 1) / TX) * ((ny + tye - 1) / tye) * nz;
}

int cubic_resident_ctas(int prec, int pass, int rows)
{
    int n = 0;
    cudaError_t e;
    if (prec == SP_F32 && rows == 2)
        e = pass == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cubic<float, SP_HEUN, 0, 1, false, false, 2>, TX * TY, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cubic<float, SP_HEUN, 1, 1, false, false, 2>, TX * TY, 0);
    else if (pass == 0)
        e = prec == SP_F64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cubic<double, SP_HEUN, 0, 1, false, false, 1>, TX * TY, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cubic<float, SP_HEUN, 0, 1, false, false, 1>, TX * TY, 0);
    else
        e = prec == SP_F64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cubic<double, SP_HEUN, 1, 1, false, false, 1>, TX * TY, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cubic<float, SP_HEUN, 1, 1, false, false, 1>, TX * TY, 0);
    return (e == cudaSuccess && n > 0) ? n : 1;
}

template cudaError_t launch_cubic<float>(int, int, const CubicParams<float> &, const float4 *, float4 *, float4 *,
                                         float4 *, const float4 *, const LlgConst<float> &, int, cudaStream_t, int,
                                         bool);
template cudaError_t launch_cubic<double>(int, int, const CubicParams<double> &, const dq4 *, dq4 *, dq4 *, dq4 *,
                                          const dq4 *, const LlgConst<double> &, int, cudaStream_t, int, bool);

}  // namespace spgb
