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
#include "internal.h"
#include "cubic.h"

namespace spgb {

namespace {

constexpr int TX = 32, TY = 8;
constexpr int HX = TX + 2, HY = TY + 2, HN = HX * HY;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename T> struct TileRec;
template <> struct TileRec<float> { using type = float4; };
template <> struct TileRec<double> { using type = dq4; };

// stage plane z (with halo) into `tile`; out-of-lattice entries are zero
template <typename T>
__device__ __forceinline__ void load_plane(const CubicParams<T> &P, const rec_t<T> *__restrict__ src, rec_t<T> *tile,
                                           int x0, int y0, int z)
{
    bool zin = true;
    if (P.per2) {
        z %= P.nz;
        z += z < 0 ? P.nz : 0;
    } else {
        zin = z >= 0 && z < P.nz;
    }
    for (int e = threadIdx.x; e < HN; e += TX * TY) {
        int hx = e % HX, hy = e / HX;
        int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
        bool in = zin;
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
        if (in) {
            const rec_t<T> *g = src + ((long)z * P.ny + gy) * P.nx + gx;
            if (sizeof(rec_t<T>) == 16) {
                cp_async16(tile + e, g);
            } else {
                cp_async16(tile + e, g);
                cp_async16(reinterpret_cast<char *>(tile + e) + 16, reinterpret_cast<const char *>(g) + 16);
            }
        } else {
            rec_t<T> zero{};
            tile[e] = zero;
        }
    }
}

template <typename T> __device__ __forceinline__ v3<T> tl(const rec_t<T> *tile, int hx, int hy)
{
    return ldc(tile, hy * HX + hx);
}

// per-plane column summary: centre, in-plane face sum, in-plane corner sum,
// in-plane face DMI field
template <typename T> struct Col {
    v3<T> c, f, k, dm;
};

template <typename T>
__device__ __forceinline__ Col<T> column(const CubicParams<T> &P, const rec_t<T> *tile, int tx, int ty)
{
    int hx = tx + 1, hy = ty + 1;
    Col<T> r;
    r.c = tl<T>(tile, hx, hy);
    v3<T> xp = tl<T>(tile, hx + 1, hy), xm = tl<T>(tile, hx - 1, hy);
    v3<T> yp = tl<T>(tile, hx, hy + 1), ym = tl<T>(tile, hx, hy - 1);
    r.f = (xp + xm) + (yp + ym);
    r.k = (tl<T>(tile, hx + 1, hy + 1) + tl<T>(tile, hx - 1, hy - 1)) +
          (tl<T>(tile, hx + 1, hy - 1) + tl<T>(tile, hx - 1, hy + 1));
    r.dm = cross(xp - xm, mk(P.Dx[0], P.Dx[1], P.Dx[2])) + cross(yp - ym, mk(P.Dy[0], P.Dy[1], P.Dy[2]));
    return r;
}

// Full local field of the middle plane m from planes lo (z-1), m, hi (z+1).
template <typename T>
__device__ __forceinline__ v3<T> field_mid(const CubicParams<T> &P, const Col<T> &lo, const Col<T> &m, const Col<T> &hi)
{
    v3<T> s1 = m.f + (lo.c + hi.c);
    v3<T> s2 = m.k + (lo.f + hi.f);
    v3<T> s3 = lo.k + hi.k;
    v3<T> B = axpy(P.J1, s1, axpy(P.J2, s2, P.J3 * s3));
    B = B + m.dm + cross(hi.c - lo.c, mk(P.Dz[0], P.Dz[1], P.Dz[2]));
    v3<T> Kh = mk(P.Kh[0], P.Kh[1], P.Kh[2]);
    T kn = T(2) * P.K * dot(Kh, m.c);
    return axpy(kn, Kh, B + mk(P.Bz[0], P.Bz[1], P.Bz[2]));
}

// PASS 0: predictor on n; PASS 1: corrector on np (q folded term, n out).
template <typename T, int SOLVER, int PASS>
__global__ void __launch_bounds__(TX *TY) k_cubic(const __grid_constant__ CubicParams<T> P, const rec_t<T> *__restrict__ src,
                                                  rec_t<T> *__restrict__ np, rec_t<T> *__restrict__ q,
                                                  rec_t<T> *__restrict__ nout, const rec_t<T> *__restrict__ Bdd,
                                                  const LlgConst<T> c, int ZC)
{
    __shared__ __align__(32) rec_t<T> tiles[2][HN];
    int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * ZC;
    int x = x0 + tx, y = y0 + ty;
    bool own = x < P.nx && y < P.ny;
    int zend = min(z0 + ZC, P.nz);
    // Pipeline: plane p lives in tiles[(p - z0 + 1) & 1].  Before the output
    // of plane z the columns of planes z-1 (lo) and z (mid) are in registers
    // and plane z+1 is in flight; plane z+2 is fetched while plane z is
    // finished.
    load_plane<T>(P, src, tiles[0], x0, y0, z0 - 1);
    cp_async_commit();
    load_plane<T>(P, src, tiles[1], x0, y0, z0);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    Col<T> lo = column<T>(P, tiles[0], tx, ty);
    __syncthreads();
    load_plane<T>(P, src, tiles[0], x0, y0, z0 + 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    Col<T> mid = column<T>(P, tiles[1], tx, ty);
    for (int z = z0; z < zend; ++z) {
        rec_t<T> *bnext = tiles[(z - z0) & 1];      // plane z+1 (in flight)
        rec_t<T> *bfree = tiles[(z - z0 + 1) & 1];  // plane z, already summarised
        cp_async_wait<0>();
        __syncthreads();
        if (z + 2 <= zend) {
            load_plane<T>(P, src, bfree, x0, y0, z + 2);
            cp_async_commit();
        }
        Col<T> hi = column<T>(P, bnext, tx, ty);
        if (own) {
            long i = ((long)z * P.ny + y) * P.nx + x;
            v3<T> B = field_mid<T>(P, lo, mid, hi);
            if (Bdd) B = B + ld(Bdd, i);
            if (PASS == 0) {
                v3<T> ni = mid.c;
                v3<T> Bth = mk(T(0), T(0), T(0));
                if (c.thermal) Bth = c.sig[0] * box_muller(thermal_bits(c.seed, c.step, c.replica, (uint32_t)i), T(0));
                v3<T> A = llg_A(c.cA[0], c.alpha, ni, B + Bth);
                if (SOLVER == SP_HEUN) {
                    v3<T> f = cross(ni, A);
                    v3<T> p = normalised(axpy(c.dt, f, ni));
                    v3<T> g = cross(p, llg_A(c.cA[0], c.alpha, p, Bth));
                    st(np, i, p);
                    st(q, i, axpy(T(0.5) * c.dt, f + g, ni));
                } else {
                    v3<T> p = rotate(ni, A, c.dt);
                    st(np, i, p);
                    st(q, i, T(0.5) * (A + llg_A(c.cA[0], c.alpha, p, Bth)));
                }
            } else {
                v3<T> p = mid.c;
                v3<T> Ap = llg_A(c.cA[0], c.alpha, p, B);
                v3<T> qi = ld(q, i);
                if (SOLVER == SP_HEUN) {
                    st(nout, i, normalised(axpy(T(0.5) * c.dt, cross(p, Ap), qi)));
                } else {
                    st(nout, i, rotate(ldc(nout, i), axpy(T(0.5), Ap, qi), c.dt));
                }
            }
        }
        lo = mid;
        mid = hi;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_cubic(int pass, int solver, const CubicParams<T> &P, const rec_t<T> *src, rec_t<T> *np, rec_t<T> *q,
                         rec_t<T> *nout, const rec_t<T> *Bdd, const LlgConst<T> &c, int zc, cudaStream_t st)
{
    dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY, (P.nz + zc - 1) / zc);
    if (pass == 0) {
        if (solver == SP_HEUN)
            k_cubic<T, SP_HEUN, 0><<<grid, TX * TY, 0, st>>>(P, src, np, q, nout, Bdd, c, zc);
        else
            k_cubic<T, SP_DEPONDT, 0><<<grid, TX * TY, 0, st>>>(P, src, np, q, nout, Bdd, c, zc);
    } else {
        if (solver == SP_HEUN)
            k_cubic<T, SP_HEUN, 1><<<grid, TX * TY, 0, st>>>(P, src, np, q, nout, Bdd, c, zc);
        else
            k_cubic<T, SP_DEPONDT, 1><<<grid, TX * TY, 0, st>>>(P, src, np, q, nout, Bdd, c, zc);
    }
    return cudaGetLastError();
}

template cudaError_t launch_cubic<float>(int, int, const CubicParams<float> &, const float4 *, float4 *, float4 *,
                                         float4 *, const float4 *, const LlgConst<float> &, int, cudaStream_t);
template cudaError_t launch_cubic<double>(int, int, const CubicParams<double> &, const dq4 *, dq4 *, dq4 *, dq4 *,
                                          const dq4 *, const LlgConst<double> &, int, cudaStream_t);

}  // namespace spgb
