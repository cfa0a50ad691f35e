// One-pass leapfrog step for the deep interior, fed by TMA (sm_103a).
//
// fused_interior computes, in a single sweep over z,
//   H^{n+1/2} = H^{n-1/2} + dt/mu  (D- E^n)          on I_H = [3, n-2]^3
//   E^{n+1}   = E^n      + dt/eps (D+ H^{n+1/2} - J) on I_E = [3, n-3]^3
// where every difference is the two-point interior row of the Appendix
// operators and no SAT applies (Eqs. (7)-(12), Algs. 1-2 interior loops).
// Reading E^n, H^{n-1/2} and eps_r once and writing H^{n+1/2}, E^{n+1} once
// moves 13 words per cell instead of the 18 + 1 of two separate half-step
// kernels.  Because H^{n+1/2} of a neighbouring tile is needed before that
// tile has written it, the new fields go to a second buffer set (ping-pong)
// and each CTA recomputes the one-node H halo it needs.
//
// A tile is W H columns x0..x0+W-1 (W = 64 or 128) by R rows y0..y0+R-1.
// Each row is served by W/64 warps, each lane by two columns of its warp's
// 64 (x0+g+L and x0+g+32+L); E is produced for the inner (W-1) x (R-1).
// Wider tiles read longer contiguous row segments and fewer halo columns per
// cell.  A 4-stage pipeline of 3D TMA tensor copies (one box per field per
// z-plane, completion on an mbarrier) keeps three planes in flight; H^{n+1/2}
// of the current and next plane is exchanged through shared memory.
//
// band_h / band_e evaluate the remaining nodes (the three boundary layers of
// each axis, closure rows and SAT penalties) with the general-path code of
// kernels.cuh, reading the old set and writing the new one.
#pragma once
#include <cuda.h>

#include "kernels.cuh"

namespace sbp {

constexpr int kFTX = 64;                 // H footprint width of the default tile and of batches
constexpr int kFTY = 8;                  // H footprint rows of the default tile and of batches
#ifndef SBP_FUSED_STAGES
#define SBP_FUSED_STAGES 4
#endif
constexpr int kStages = SBP_FUSED_STAGES;     // TMA pipeline depth (planes in shared memory)
constexpr unsigned kWaitLimit = 1u << 22;

constexpr int round128(int bytes) { return (bytes + 127) / 128 * 128; }

// Shared-memory geometry of one pipeline stage for field storage type S and
// a tile of R H rows by W columns (E is produced on the inner R-1 rows).  A
// TMA box starts at an x that is a multiple of 16 bytes (4 FP32 or 8 FP16
// elements) at or below x0-1 and spans the W columns after it: kBX columns.
// The E box holds rows y0-1 .. y0+R-1, the H and eps boxes rows y0 .. y0+R-1.
// The eps box (always FP32) uses the same start and width.
template <typename S, int R = kFTY, int W = kFTX>
struct FusedGeom {
    static_assert(W == 64 || W == 128, "tile width");
    static constexpr int kWarps = R * (W / 64);
    static constexpr int kERows = R + 1;
    static constexpr int kHRows = R;
    static constexpr int kHbufFloats = 2 * 3 * R * W;      // H^{n+1/2} of two planes
    static constexpr int kAlign = 16 / (int)sizeof(S);
    static constexpr int kBX = W + kAlign;
    static constexpr int kEBytes = round128(kERows * kBX * (int)sizeof(S));   // one E box slot
    static constexpr int kHBytes = round128(kHRows * kBX * (int)sizeof(S));   // one H box slot
    static constexpr int kPBytes = round128(kHRows * kBX * 4);                // the eps box slot
    static constexpr int kStageBytes = 3 * kEBytes + 3 * kHBytes + kPBytes;
    static constexpr int kTxBytes = (3 * kERows + 3 * kHRows) * kBX * (int)sizeof(S) + kHRows * kBX * 4;
    static constexpr int kSmem = kStages * kStageBytes + kHbufFloats * 4 + kStages * 8;
};
constexpr int kFusedSmem = FusedGeom<float>::kSmem;

template <typename S>
struct FusedParamsT {
    S *out[6];                           // new set: element (i,j,k) at k*sz + j*sy + i
    float pscale[2];                     // probe value = stored value * pscale[E=0 / H=1]
    int n[3];
    long long sy, sz;
    Coef<float> B[3], A[3], AJ;
    double dt;
    int nsrc, nprb;
    Src src[kMaxSources];
    Prb prb[kMaxProbes];
    float *probe_buf;
    long long probe_cap, probe_slot, step;
    int kchunk;
    int *error_flag;                     // set to 1 when a pipeline wait gives up
    unsigned wait_limit;                 // polls before a pipeline wait gives up
    int test_stall;                      // test hook: issue no plane loads, so every wait runs out
};
using FusedParams = FusedParamsT<float>;

// --- mbarrier / TMA helpers (inline PTX) ----------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase did not complete within `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned limit = kWaitLimit)
{
    for (unsigned it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
// Orders this thread's earlier shared-memory reads (generic proxy) before the
// TMA copies (async proxy) that the next CTA barrier releases into the stage
// they read.  A warp passes a barrier with a load still outstanding when the
// value is first used after the barrier; the copy could then overwrite the
// slot before the load reads it.  Within a block that happens only to the
// carries read before the plane loop (E of plane k0-1) and to the eps cells
// of its first plane (no E update yet): every other value read from a stage
// feeds a store issued before that plane's barrier.
__device__ __forceinline__ void fence_generic_to_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

struct FusedMaps {
    CUtensorMap e[3], h[3], eps;
};

template <typename S, int R, int W>
__device__ __forceinline__ void issue_plane(const FusedMaps &m, unsigned char *stage, uint64_t *bar, int xb, int y0,
                                            int plane)
{
    using Gm = FusedGeom<S, R, W>;
    mbar_expect_tx(bar, Gm::kTxBytes);
#pragma unroll
    for (int f = 0; f < 3; ++f) tma_load_3d(stage + f * Gm::kEBytes, &m.e[f], xb, y0 - 1, plane, bar);
#pragma unroll
    for (int f = 0; f < 3; ++f) tma_load_3d(stage + 3 * Gm::kEBytes + f * Gm::kHBytes, &m.h[f], xb, y0, plane, bar);
    tma_load_3d(stage + 3 * Gm::kEBytes + 3 * Gm::kHBytes, &m.eps, xb, y0, plane, bar);
}

// One CTA of the one-pass interior step: tile (bx, by) in x/y, z-chunk bz,
// time step `step` (J is evaluated at t^{step+1/2}), probe sample `pslot`.
// A value rounded to the storage type once: the FP32 value later arithmetic
// reads (FP16 storage: the stored half, widened) and the stored element.
template <typename S> struct Rounded { float f; S s; };
template <typename S>
__device__ __forceinline__ Rounded<S> rounded(float v)
{
    if constexpr (std::is_same<S, __half>::value) {
        const __half h = __float2half_rn(v);
        return {__half2float(h), h};
    } else {
        return {v, v};
    }
}

template <bool SRC, typename S, int R = kFTY, int W = kFTX>
__device__ __forceinline__ void fused_body(const FusedMaps &maps, const FusedParamsT<S> &p, long long step,
                                           long long pslot, int bx, int by, int bz, unsigned char *smem)
{
    using Gm = FusedGeom<S, R, W>;
    constexpr int kFTY = R;                        // tile rows of this instantiation
    constexpr int kFTX = W;                        // tile columns
    constexpr int kGroups = W / 64;                // warps per row
    constexpr int kBX = Gm::kBX;
    float *hbuf = reinterpret_cast<float *>(smem + kStages * Gm::kStageBytes);
    uint64_t *bar = reinterpret_cast<uint64_t *>(hbuf + Gm::kHbufFloats);
    // slots of a stage: E fields, H fields (storage type), eps (FP32)
    auto slotE = [&](int st, int f) { return reinterpret_cast<const S *>(smem + st * Gm::kStageBytes + f * Gm::kEBytes); };
    auto slotH = [&](int st, int f) {
        return reinterpret_cast<const S *>(smem + st * Gm::kStageBytes + 3 * Gm::kEBytes + f * Gm::kHBytes);
    };
    auto slotP = [&](int st) {
        return reinterpret_cast<const float *>(smem + st * Gm::kStageBytes + 3 * Gm::kEBytes + 3 * Gm::kHBytes);
    };

    // warp wid serves row w, columns cg .. cg+63 of the tile
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int w = wid / kGroups, cg = (wid % kGroups) * 64;
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    const int x0 = 3 + bx * (kFTX - 1);
    const int y0 = 3 + by * (kFTY - 1);
    const int k0 = 3 + bz * p.kchunk;
    const int k1 = min(k0 + p.kchunk, nz - 2);       // E planes [k0, k1); H planes [k0, k1]
    const int xb = (x0 - 1) & ~(Gm::kAlign - 1);
    const int cx0 = x0 - xb;                          // smem column of x0, in 1..kAlign
    const int nplanes = k1 - k0 + 2;                  // planes k0-1 .. k1 are loaded
    const int j = y0 + w;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int issued = 0;                                   // planes issued (thread 0's count)
    if (threadIdx.x == 0 && !p.test_stall)
        for (; issued < kStages && issued < nplanes; ++issued)
            issue_plane<S, R, W>(maps, smem + issued * Gm::kStageBytes, &bar[issued], xb, y0, k0 - 1 + issued);
    // J(t^{n+1/2}) of every source is the same at each node it reaches, so
    // warp 1 evaluates it once per CTA (FP64 waveform, rounded to FP32 once)
    // while the first planes load; it is first read after the barrier below.
    static_assert(kMaxSources <= 32, "one lane of warp 1 per source");
    __shared__ float sJ[kMaxSources];
    if (SRC && wid == 1 && lane < p.nsrc) {
        const Src &Sr = p.src[lane];
        const double t_half = ((double)step + 0.5) * p.dt;
        sJ[lane] = (float)(Sr.amp * waveform(Sr.wf, t_half, Sr.tw, Sr.t0, Sr.f));
    }

    // per-thread probe / source masks for the two columns
    unsigned long long pmask[2] = {0ull, 0ull};
    unsigned smask[2] = {0u, 0u};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = x0 + cg + lane + 32 * h;
        for (int q = 0; q < p.nprb; ++q)
            if (p.prb[q].i == i && p.prb[q].j == j) pmask[h] |= 1ull << q;
        if (SRC)
            for (int q = 0; q < p.nsrc; ++q)
                if ((p.src[q].i < 0 || p.src[q].i == i) && (p.src[q].j < 0 || p.src[q].j == j)) smask[h] |= 1u << q;
    }
    const bool rowE = w < kFTY - 1 && j <= ny - 3;
    const bool rowH = j <= ny - 2 && (w < kFTY - 1 || j == ny - 2);
    // per column: stores owned (H) / produced (E) by this thread, and the
    // column's offset within a plane
    bool colH[2], colE[2];
    int obase[2];                                     // j * sy + i (a plane has fewer than 2^31 elements)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = cg + lane + 32 * h, i = x0 + c;
        colH[h] = rowH && i <= nx - 2 && (c < kFTX - 1 || i == nx - 2);
        colE[h] = rowE && c < kFTX - 1 && i <= nx - 3;
        obase[h] = j * (int)p.sy + i;
    }
    const Coef<float> Bx = p.B[0], By = p.B[1], Bz = p.B[2];
    const Coef<float> Ax = p.A[0], Ay = p.A[1], Az = p.A[2];

    bool ok = true;
    bool aborted = false;
    int waited = 0;                                   // load index of the next plane to wait for
    // register carries of the previous plane (own columns): E^n, H^{n+1/2} and
    // the eps cells (rows j, j+1; columns i, i+1) of that plane
    float ec[2][3], hc[2][3], epc[2][3];
    if (nplanes > 0) { ok = mbar_wait_bounded(&bar[0], 0, p.wait_limit); waited = 1; }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int re = (w + 1) * kBX + cx0 + cg + lane + 32 * h;
#pragma unroll
        for (int f = 0; f < 3; ++f) { ec[h][f] = ld_s(slotE(0, f) + re); hc[h][f] = 0.f; }
#pragma unroll
        for (int f = 0; f < 3; ++f) epc[h][f] = 0.f;
    }
    fence_generic_to_async();                         // the E carries of plane k0-1
    if (__syncthreads_or(!ok)) aborted = true;
    if (!aborted && threadIdx.x == 0 && kStages < nplanes) {   // plane k0-1 is in registers now
        issue_plane<S, R, W>(maps, smem, &bar[0], xb, y0, k0 - 1 + kStages);
        ++issued;
    }
#pragma unroll(sizeof(S) == 4 ? 2 : 1)   // two planes per iteration with FP32 storage (faster there, slower with FP16)
    for (int q = k0; q <= k1 && !aborted; ++q) {
        const int iq = q - k0 + 1;                   // load index of plane q
        const int sq = iq % kStages;
        if (ok) ok = mbar_wait_bounded(&bar[sq], (iq / kStages) & 1, p.wait_limit);
        waited = iq + 1;
        const S *E0 = slotE(sq, 0), *E1 = slotE(sq, 1), *E2 = slotE(sq, 2);   // plane q
        const S *H0 = slotH(sq, 0), *H1 = slotH(sq, 1), *H2 = slotH(sq, 2);
        const float *eq = slotP(sq);
        float *Hq = hbuf + (q & 1) * (3 * kFTY * kFTX);
        const float *Hp = hbuf + ((q - 1) & 1) * (3 * kFTY * kFTX);
        const bool doE = q > k0;
        const int pl = q - 1;
        // sources acting on E plane pl, looked up only by threads whose
        // columns some source reaches
        unsigned splane = 0u;
        if (SRC && (smask[0] | smask[1]))
            for (int b = 0; b < p.nsrc; ++b)
                if (p.src[b].k < 0 || p.src[b].k == pl) splane |= 1u << b;

        // output rows of plane q (H) and pl (E): a base shared by the CTA plus the
        // thread's 32-bit offset within the plane
        S *const oH0 = p.out[3] + (long long)q * p.sz, *const oH1 = p.out[4] + (long long)q * p.sz,
                 *const oH2 = p.out[5] + (long long)q * p.sz;
        S *const oE0 = p.out[0] + (long long)pl * p.sz, *const oE1 = p.out[1] + (long long)pl * p.sz,
                 *const oE2 = p.out[2] + (long long)pl * p.sz;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = cg + lane + 32 * h;
            const int cc = cx0 + c;
            // ---- H^{n+1/2} at (i, j, q) --------------------------------------
            const int re = (w + 1) * kBX + cc;            // E slot row of j
            const int rh = w * kBX + cc;                  // H slot row of j
            const float exq = ld_s(E0 + re), ex_jm = ld_s(E0 + re - kBX);
            const float eyq = ld_s(E1 + re), ey_im = ld_s(E1 + re - 1);
            const float ezq = ld_s(E2 + re), ez_im = ld_s(E2 + re - 1), ez_jm = ld_s(E2 + re - kBX);
            typename AccOf<float, S>::type bx, by, bz;
            bx.add(Bz, eyq - ec[h][1]); bx.add(By, ezq - ez_jm, -1.f);
            by.add(Bx, ezq - ez_im);    by.add(Bz, exq - ec[h][0], -1.f);
            bz.add(By, exq - ex_jm);    bz.add(Bx, eyq - ey_im, -1.f);
            // the values the stores keep (FP16 storage rounds here, and E
            // below uses the rounded H, as a separate E half-step would)
            const Rounded<S> rhx = rounded<S>(ld_s(H0 + rh) + plain_increment(bx));
            const Rounded<S> rhy = rounded<S>(ld_s(H1 + rh) + plain_increment(by));
            const Rounded<S> rhz = rounded<S>(ld_s(H2 + rh) + plain_increment(bz));
            const float hx = rhx.f, hy = rhy.f, hz = rhz.f;
            Hq[(0 * kFTY + w) * kFTX + c] = hx;
            Hq[(1 * kFTY + w) * kFTX + c] = hy;
            Hq[(2 * kFTY + w) * kFTX + c] = hz;
            if (colH[h] && (q < k1 || q == nz - 2)) {
                oH0[obase[h]] = rhx.s;
                oH1[obase[h]] = rhy.s;
                oH2[obase[h]] = rhz.s;
                if (pmask[h]) {
                    unsigned long long m = pmask[h];
                    while (m) {
                        const int b = __ffsll(m) - 1;
                        m &= m - 1;
                        const Prb &P = p.prb[b];
                        if (P.k == q && P.comp >= 3 && pslot < p.probe_cap)
                            p.probe_buf[(long long)b * p.probe_cap + pslot] =
                                (P.comp == 3 ? hx : P.comp == 4 ? hy : hz) * p.pscale[1];
                    }
                }
            }
            // eps cells of plane q (rows j, j+1; columns i, i+1), as the pair sums
            // the node sums of cell_sum are built from: (a+b)+(c+d)
            const int r0 = w * kBX + cc, r1 = r0 + kBX;
            const float q00 = eq[r0], q01 = eq[r1], q10 = eq[r0 + 1], q11 = eq[r1 + 1];
            const float qa = q00 + q01, qb = q00 + q10, qc = q01 + q11;

            // ---- E^{n+1} at (i, j, q-1): neighbours' H of plane q-1 from shared
            // memory (written last iteration), own H of planes q-1, q from registers
            if (doE && colE[h]) {
                const float hx_jp = Hp[(0 * kFTY + w + 1) * kFTX + c];
                const float hy_ip = Hp[(1 * kFTY + w) * kFTX + c + 1];
                const float hz_ip = Hp[(2 * kFTY + w) * kFTX + c + 1];
                const float hz_jp = Hp[(2 * kFTY + w + 1) * kFTX + c];
                const float hxp = hc[h][0], hyp = hc[h][1], hzp = hc[h][2];
                typename AccOf<float, S>::type ax, ay, az;
                ax.add(Ay, hz_jp - hzp); ax.add(Az, hy - hyp, -1.f);
                ay.add(Az, hx - hxp);    ay.add(Ax, hz_ip - hzp, -1.f);
                az.add(Ax, hy_ip - hyp); az.add(Ay, hx_jp - hxp, -1.f);
                // node sums in the association of cell_sum:
                //   Ex (m + m_y) + (m_z + m_yz), Ey (m + m_x) + (m_z + m_xz), Ez (m + m_x) + (m_y + m_xy)
                const float sx = epc[h][0] + qa;
                const float sy = epc[h][1] + qb;
                const float sz = epc[h][1] + epc[h][2];
                if (SRC && (smask[h] & splane)) {
                    unsigned m = smask[h] & splane;
                    while (m) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1;
                        const float J = sJ[b];
                        const int comp = p.src[b].comp;
                        if (comp == 0) ax.add(p.AJ, J, -1.f);
                        else if (comp == 1) ay.add(p.AJ, J, -1.f);
                        else az.add(p.AJ, J, -1.f);
                    }
                }
                const Rounded<S> rex = rounded<S>(ec[h][0] + scaled_increment(ax, sx));
                const Rounded<S> rey = rounded<S>(ec[h][1] + scaled_increment(ay, sy));
                const Rounded<S> rez = rounded<S>(ec[h][2] + scaled_increment(az, sz));
                const float ex = rex.f, ey = rey.f, ez = rez.f;
                oE0[obase[h]] = rex.s;
                oE1[obase[h]] = rey.s;
                oE2[obase[h]] = rez.s;
                if (pmask[h]) {
                    unsigned long long m = pmask[h];
                    while (m) {
                        const int b = __ffsll(m) - 1;
                        m &= m - 1;
                        const Prb &P = p.prb[b];
                        if (P.k == pl && P.comp < 3 && pslot < p.probe_cap)
                            p.probe_buf[(long long)b * p.probe_cap + pslot] =
                                (P.comp == 0 ? ex : P.comp == 1 ? ey : ez) * p.pscale[0];
                    }
                }
            }
            // carry plane q
            ec[h][0] = exq; ec[h][1] = eyq; ec[h][2] = ezq;
            hc[h][0] = hx; hc[h][1] = hy; hc[h][2] = hz;
            epc[h][0] = qa; epc[h][1] = qb; epc[h][2] = qc;
        }
        // one barrier per plane: hbuf[q&1] complete, hbuf[(q-1)&1] and stage q free
        if (!doE) fence_generic_to_async();           // the eps carries of plane k0
        if (__syncthreads_or(!ok)) { aborted = true; break; }
        if (threadIdx.x == 0) {
            const int nxt = q + kStages;
            if (nxt <= k1) {
                issue_plane<S, R, W>(maps, smem + sq * Gm::kStageBytes, &bar[sq], xb, y0, nxt);
                ++issued;
            }
        }
    }
    if (aborted && threadIdx.x == 0) {
        // a pipeline wait gave up: flag it, then wait (bounded) for every copy
        // still in flight so that none lands in shared memory after exit
        atomicExch(p.error_flag, 1);
        for (int L = waited > 0 ? waited - 1 : 0; L < issued; ++L)
            (void)mbar_wait_bounded(&bar[L % kStages], (L / kStages) & 1, p.wait_limit);
    }
    // Leave the shared memory reusable by a later tile of the same CTA (the
    // persistent batched kernel): every thread's reads of the stages ordered
    // before later TMA writes, and the barriers invalidated so that they can
    // be initialised again.
    fence_generic_to_async();
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < kStages; ++s) mbar_inval(&bar[s]);
}

template <bool SRC, typename S, int R, int W>
__global__ void __launch_bounds__(FusedGeom<S, R, W>::kWarps * 32,
                                  FusedGeom<S, R, W>::kWarps >= 16 ? 1 : (kStages <= 3 ? 3 : 2))
    fused_interior(const __grid_constant__ FusedMaps maps, const FusedParamsT<S> p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    fused_body<SRC, S, R, W>(maps, p, p.step, p.probe_slot, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
}

// ---------------------------------------------------------------------------
// Band kernels: every node outside the interior box [lo, hi_a] of its phase.
// The band is split into disjoint slabs: the x-ends (i < lo or i > hi_x, every
// j and k), then the y-ends of the rest (every k), then the z-ends of the
// rest.  Work goes out by warps: a warp of the z or y slab takes up to 32
// consecutive nodes of one x-row (coalesced), a warp of the x slab 4 x-end
// nodes of 8 consecutive rows of one plane.  Every index is decoded once per
// warp, and each warp knows which axes can put its nodes on a closure row or
// a face (G); along the others its nodes are interior and take the two-point
// row, the same expression the general row evaluates there.
// ---------------------------------------------------------------------------
struct Band {
    int lo;                   // interior box lower bound (every axis)
    int hi[3];                // interior box upper bound per axis (inclusive)
    unsigned segs;            // 32-node x segments from x = 0 up to hi_x
    unsigned zplanes;         // planes of the z slab
    unsigned yrows;           // rows per plane of the y slab
    unsigned jin;             // interior rows (z slab rows per plane)
    unsigned xgroups;         // 8-row groups per plane of the x slab
    unsigned wz, wy, wx;      // warps of the three slabs
    unsigned ctas;            // CTAs of 256 threads over all warps
};

// Node of `lane` in band warp w, the warp's index box [il,ih] x [jl,jh] x {k}
// and its closure axes G (bit a).  False when the lane has no node.
__device__ __forceinline__ bool band_lane(const Band &b, const int n[3], unsigned w, int lane, int &i, int &j, int &k,
                                          int &il, int &ih, int &jl, int &jh, int &G)
{
    const int lo = b.lo;
    if (w < b.wz + b.wy) {
        const bool zs = w < b.wz;
        if (!zs) w -= b.wz;
        const unsigned r = w / b.segs;
        const unsigned seg = w - r * b.segs;
        if (zs) {
            const unsigned pl = r / b.jin;
            j = lo + (int)(r - pl * b.jin);
            k = (int)pl < lo ? (int)pl : b.hi[2] + 1 + ((int)pl - lo);
            G = 4;
        } else {
            const unsigned kk = r / b.yrows;
            const int jr = (int)(r - kk * b.yrows);
            k = (int)kk;
            j = jr < lo ? jr : b.hi[1] + 1 + (jr - lo);
            G = (k < lo || k > b.hi[2]) ? 6 : 2;
        }
        jl = jh = j;
        il = (int)seg * 32;
        ih = il + 31;
        i = il + lane;
        return i >= lo && i <= b.hi[0];
    }
    w -= b.wz + b.wy;
    const unsigned side = w & 1u, r = w >> 1;
    const unsigned kk = r / b.xgroups;
    const int g = (int)(r - kk * b.xgroups);
    k = (int)kk;
    jl = 8 * g;
    jh = min(jl + 7, n[1] + 1);
    j = jl + (lane >> 2);
    const int c = lane & 3;
    il = side ? b.hi[0] + 1 : 0;
    ih = il + 3;
    i = il + c;
    G = 1 | ((jl < lo || jh > b.hi[1]) ? 2 : 0) | ((k < lo || k > b.hi[2]) ? 4 : 0);
    return j <= jh && (side ? i <= n[0] + 1 : c < lo);
}

// Probes of components [c0, c0+2] inside the warp's box (one bit per probe).
__device__ __forceinline__ unsigned long long warp_probe_mask(const Prb *prb, int nprb, int c0, int k, int il, int ih,
                                                              int jl, int jh, int lane)
{
    unsigned long long m = 0ull;
    for (int q0 = 0; q0 < nprb; q0 += 32) {
        const int q = q0 + lane;
        bool hit = false;
        if (q < nprb) {
            const Prb P = prb[q];
            hit = P.comp >= c0 && P.comp <= c0 + 2 && P.k == k && P.j >= jl && P.j <= jh && P.i >= il && P.i <= ih;
        }
        m |= (unsigned long long)__ballot_sync(0xffffffffu, hit) << q0;
    }
    return m;
}

template <typename T, typename S>
__device__ __forceinline__ void band_probes(const Params<T, S> &p, unsigned long long m, int c0, int i, int j,
                                            long long pslot, const T v[3], const bool have[3])
{
    while (m) {
        const int q = __ffsll((long long)m) - 1;
        m &= m - 1;
        const Prb &P = p.prb[q];
        const int c = P.comp - c0;
        const bool hv = c == 0 ? have[0] : c == 1 ? have[1] : have[2];
        if (P.i == i && P.j == j && hv && pslot < p.probe_cap)
            p.probe_buf[(long long)q * p.probe_cap + pslot] = (c == 0 ? v[0] : c == 1 ? v[1] : v[2]) * p.fscale[c0 >= 3];
    }
}

// H^{n+1/2} at one band node, closure axes G: every load first (in bounds for
// all three components: the node and its row entries lie in the padded
// layout), then the updates.
template <typename T, bool MUVAR, int G, bool CG, typename S>
__device__ __forceinline__ void band_h_at(const Params<T, S> &p, const int idx[3], long long o, const bool have[3],
                                          S *const outs[3], T hn[3])
{
    Tri<T> vx[2], vy[2], vz[2];
    h_gather<T, 3, G, CG>(p, idx, o, vx);
    h_gather<T, 4, G, CG>(p, idx, o, vy);
    h_gather<T, 5, G, CG>(p, idx, o, vz);
    const T hx = ldf<CG>(p.F[3] + o), hy = ldf<CG>(p.F[4] + o), hz = ldf<CG>(p.F[5] + o);
    if (have[0]) st_s(outs[0] + o, hn[0] = quant<S>(h_apply<T, 3, MUVAR, G>(p, idx, o, hx, vx)));
    if (have[1]) st_s(outs[1] + o, hn[1] = quant<S>(h_apply<T, 4, MUVAR, G>(p, idx, o, hy, vy)));
    if (have[2]) st_s(outs[2] + o, hn[2] = quant<S>(h_apply<T, 5, MUVAR, G>(p, idx, o, hz, vz)));
}

// Yee FDTD comparator (the FDTD method the paper measures its overhead
// against, with strong PEC walls) on the same grid: H exists on the half nodes
// 1..n of its minus-grid axes (the SBP boundary nodes 0 and n+1 are not part
// of it), E on the half nodes 1..n of its minus-grid axes and the interior
// nodes 1..n-1 of its plus-grid axes (tangential E on a wall stays zero); every
// row is the two-point row and no SAT applies.  Nodes outside the Yee set keep
// their value (copied to the new set).
template <int C>
__device__ __forceinline__ bool yee_node(const int idx[3], const int n[3])
{
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        in = in && idx[a] >= 1 && idx[a] <= (on_plus(C, a) ? n[a] - 1 : n[a]);
    return in;
}

template <typename T, bool MUVAR, int C, typename S>
__device__ __forceinline__ void yee_h(const Params<T, S> &p, const int idx[3], long long o, bool have, S *out, T &hn)
{
    if (!have) return;
    const T hold = ld_s(p.F[C] + o);
    // H on its plus-grid axis is a face-normal component: nodes 0..n all exist
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (!on_plus(C, a)) in = in && idx[a] >= 1 && idx[a] <= p.n[a];
    if (in) {
        Tri<T> v[2];
        h_gather<T, C, 0>(p, idx, o, v);
        hn = quant<S>(h_apply<T, C, MUVAR, 0>(p, idx, o, hold, v));
    } else {
        hn = hold;
    }
    st_s(out + o, hn);
}

template <typename T, bool MUVAR, int C, typename S>
__device__ __forceinline__ void yee_e(const Params<T, S> &p, const int idx[3], long long o, bool have, unsigned sm,
                                      double t_half, S *out, T &en)
{
    if (!have) return;
    const T eold = ld_s(p.F[C] + o);
    if (yee_node<C>(idx, p.n)) {
        Tri<T> v[2];
        e_gather<T, C, false, 0>(p, idx, o, v);
        const T se = cell_sum<C, T>(p.eps, o, p.sy, p.sz);
        en = quant<S>(e_apply<T, C, MUVAR, false, 0>(p, idx, o, eold, se, v, sm, t_half));
    } else {
        en = eold;
    }
    st_s(out + o, en);
}

// H^{n+1/2} at the nodes of band warp w: p.F = {E^n (old), H^{n-1/2} (old)}, outs = new H.
// CG: field reads through L2 only (the persistent batched kernel, whose other
// CTAs wrote them earlier in the same launch).
template <typename T, bool MUVAR, bool CG = false, typename S>
__device__ __forceinline__ void band_h_warp(const Params<T, S> &p, const Band &b, unsigned w, int lane, long long pslot,
                                            S *const outs[3])
{
    int i, j, k, il, ih, jl, jh, G;
    const bool valid = band_lane(b, p.n, w, lane, i, j, k, il, ih, jl, jh, G);
    const unsigned long long pm = p.nprb ? warp_probe_mask(p.prb, p.nprb, 3, k, il, ih, jl, jh, lane) : 0ull;
    if (!valid) return;
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    const int idx[3] = {i, j, k};
    const long long o = (long long)k * p.sz + (long long)j * p.sy + i;
    T hn[3];
    const bool have[3] = {i <= nx && j <= ny + 1 && k <= nz + 1, i <= nx + 1 && j <= ny && k <= nz + 1,
                          i <= nx + 1 && j <= ny + 1 && k <= nz};
    if (p.fdtd) {
        yee_h<T, MUVAR, 3>(p, idx, o, have[0], outs[0], hn[0]);
        yee_h<T, MUVAR, 4>(p, idx, o, have[1], outs[1], hn[1]);
        yee_h<T, MUVAR, 5>(p, idx, o, have[2], outs[2], hn[2]);
    } else {
        switch (G) {   // uniform per warp
        case 4: band_h_at<T, MUVAR, 4, CG>(p, idx, o, have, outs, hn); break;
        case 2: band_h_at<T, MUVAR, 2, CG>(p, idx, o, have, outs, hn); break;
        case 6: band_h_at<T, MUVAR, 6, CG>(p, idx, o, have, outs, hn); break;
        case 1: band_h_at<T, MUVAR, 1, CG>(p, idx, o, have, outs, hn); break;
        default: band_h_at<T, MUVAR, 7, CG>(p, idx, o, have, outs, hn); break;
        }
    }
    if (pm) band_probes(p, pm, 3, i, j, pslot, hn, have);
}

// At most 56 registers: two 256-thread CTAs then fit on an SM beside a 512-thread
// one-pass CTA (band H runs concurrently with it), without spills.
template <typename T, bool MUVAR, typename S>
__global__ void __maxnreg__(56) band_h(const Params<T, S> p, const Band b, S *hx_out, S *hy_out, S *hz_out)
{
    const unsigned w = blockIdx.x * 8u + (threadIdx.x >> 5);
    if (w >= b.wz + b.wy + b.wx) return;
    S *const outs[3] = {hx_out, hy_out, hz_out};
    band_h_warp<T, MUVAR>(p, b, w, threadIdx.x & 31, p.probe_slot, outs);
}

// E^{n+1} at one band node, closure axes G (see band_h_at).
template <typename T, bool MUVAR, int G, bool CG, typename S>
__device__ __forceinline__ void band_e_at(const Params<T, S> &p, const int idx[3], long long o, const bool have[3],
                                          unsigned sm, double t_half, S *const outs[3], T en[3])
{
    Tri<T> vx[2], vy[2], vz[2];
    e_gather<T, 0, CG, G>(p, idx, o, vx);
    e_gather<T, 1, CG, G>(p, idx, o, vy);
    e_gather<T, 2, CG, G>(p, idx, o, vz);
    const T ex = ldf<CG>(p.F[0] + o), ey = ldf<CG>(p.F[1] + o), ez = ldf<CG>(p.F[2] + o);
    const T sx = cell_sum<0, T>(p.eps, o, p.sy, p.sz);
    const T sy = cell_sum<1, T>(p.eps, o, p.sy, p.sz);
    const T sz = cell_sum<2, T>(p.eps, o, p.sy, p.sz);
    if (have[0]) st_s(outs[0] + o, en[0] = quant<S>(e_apply<T, 0, MUVAR, false, G>(p, idx, o, ex, sx, vx, sm, t_half)));
    if (have[1]) st_s(outs[1] + o, en[1] = quant<S>(e_apply<T, 1, MUVAR, false, G>(p, idx, o, ey, sy, vy, sm, t_half)));
    if (have[2]) st_s(outs[2] + o, en[2] = quant<S>(e_apply<T, 2, MUVAR, false, G>(p, idx, o, ez, sz, vz, sm, t_half)));
}

// E^{n+1} at the nodes of band warp w: p.F = {E^n (old), H^{n+1/2} (new)}, outs = new E.
template <typename T, bool MUVAR, bool CG = false, typename S>
__device__ __forceinline__ void band_e_warp(const Params<T, S> &p, const Band &b, unsigned w, int lane, long long step,
                                            long long pslot, S *const outs[3])
{
    int i, j, k, il, ih, jl, jh, G;
    const bool valid = band_lane(b, p.n, w, lane, i, j, k, il, ih, jl, jh, G);
    const unsigned long long pm = p.nprb ? warp_probe_mask(p.prb, p.nprb, 0, k, il, ih, jl, jh, lane) : 0ull;
    // sources that can reach the warp's box (point, line or sheet), then this node's
    unsigned wm = 0u;
    if (p.nsrc) {
        bool hit = false;
        if (lane < p.nsrc) {
            const Src &Sr = p.src[lane];
            hit = (Sr.i < 0 || (Sr.i >= il && Sr.i <= ih)) && (Sr.j < 0 || (Sr.j >= jl && Sr.j <= jh)) &&
                  (Sr.k < 0 || Sr.k == k);
        }
        wm = __ballot_sync(0xffffffffu, hit);
    }
    if (!valid) return;
    unsigned sm = 0u;
    for (unsigned m = wm; m; m &= m - 1) {
        const int q = __ffs(m) - 1;
        if ((p.src[q].i < 0 || p.src[q].i == i) && (p.src[q].j < 0 || p.src[q].j == j)) sm |= 1u << q;
    }
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    const int idx[3] = {i, j, k};
    const long long o = (long long)k * p.sz + (long long)j * p.sy + i;
    const double t_half = ((double)step + 0.5) * p.dt;
    T en[3];
    const bool have[3] = {i <= nx + 1 && j <= ny && k <= nz, i <= nx && j <= ny + 1 && k <= nz,
                          i <= nx && j <= ny && k <= nz + 1};
    if (p.fdtd) {
        yee_e<T, MUVAR, 0>(p, idx, o, have[0], sm, t_half, outs[0], en[0]);
        yee_e<T, MUVAR, 1>(p, idx, o, have[1], sm, t_half, outs[1], en[1]);
        yee_e<T, MUVAR, 2>(p, idx, o, have[2], sm, t_half, outs[2], en[2]);
    } else {
        switch (G) {   // uniform per warp
        case 4: band_e_at<T, MUVAR, 4, CG>(p, idx, o, have, sm, t_half, outs, en); break;
        case 2: band_e_at<T, MUVAR, 2, CG>(p, idx, o, have, sm, t_half, outs, en); break;
        case 6: band_e_at<T, MUVAR, 6, CG>(p, idx, o, have, sm, t_half, outs, en); break;
        case 1: band_e_at<T, MUVAR, 1, CG>(p, idx, o, have, sm, t_half, outs, en); break;
        default: band_e_at<T, MUVAR, 7, CG>(p, idx, o, have, sm, t_half, outs, en); break;
        }
    }
    if (pm) band_probes(p, pm, 0, i, j, pslot, en, have);
}

template <typename T, bool MUVAR, typename S>
__global__ void __launch_bounds__(256, 4) band_e(const Params<T, S> p, const Band b, S *ex_out, S *ey_out, S *ez_out)
{
    const unsigned w = blockIdx.x * 8u + (threadIdx.x >> 5);
    if (w >= b.wz + b.wy + b.wx) return;
    S *const outs[3] = {ex_out, ey_out, ez_out};
    band_e_warp<T, MUVAR>(p, b, w, threadIdx.x & 31, p.step, p.probe_slot, outs);
}

// ---------------------------------------------------------------------------
// Batched step: one launch per kernel kind advances every grid of a batch
// (continuous batching of many simulations).  A CTA finds its grid in a
// prefix table of CTA counts; the grid's parameters and TMA maps live in
// global memory; the step index comes from a device counter, so a captured
// chunk of K steps can be replayed (the launches of a chunk carry offsets
// 0..K-1 and batch_advance adds the steps taken).  Grids that reached their
// target step skip their work, so a chunk may end a grid early.
// ---------------------------------------------------------------------------
struct BatchGrid {
    FusedMaps maps[2];            // TMA maps reading field set 0 / set 1
    FusedParams fp[2];            // fp[c]: reads set c, writes set c^1
    Params<float> ph[2];          // band H, current set c
    Params<float> pe[2];          // band E: E of set c, H of set c^1
    float *hout[2][3], *eout[2][3];   // new-set outputs when the current set is c
    Band bh, be;
    long long *counter;           // steps taken (device)
    long long target;             // the grid stops when the counter reaches this
    long long cstart;             // counter value at which the current set was cur0
    long long probe_base;
    int cur0;
    int tiles[3];
};

__device__ __forceinline__ int find_slot(const int *pre, int n, int b)
{
    int lo = 0, hi = n - 1;                 // largest g with pre[g] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool batch_state(const BatchGrid &g, int offset, long long &step, int &par)
{
    step = *g.counter + offset;
    if (step >= g.target) return false;
    par = (g.cur0 + (int)((step - g.cstart) & 1)) & 1;
    return true;
}

// R: tile rows of every member's one-pass tiles (8, or 16 when every member
// has a full 16-row tile).
template <int R>
__global__ void __launch_bounds__(R * 32, R >= 16 ? 1 : (kStages <= 3 ? 3 : 2))
    fused_batched(const BatchGrid *G, const int *pre, int n, int offset)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int g = find_slot(pre, n, blockIdx.x);
    const BatchGrid &B = G[g];
    long long step;
    int par;
    if (!batch_state(B, offset, step, par)) return;
    const int local = blockIdx.x - pre[g];
    const int tx = B.tiles[0], ty = B.tiles[1];
    fused_body<true, float, R>(B.maps[par], B.fp[par], step, step - B.probe_base, local % tx, (local / tx) % ty,
                               local / (tx * ty), smem_raw);
}

__global__ void __launch_bounds__(256) band_h_batched(const BatchGrid *G, const int *pre, int n, int offset)
{
    const int g = find_slot(pre, n, blockIdx.x);
    const BatchGrid &B = G[g];
    long long step;
    int par;
    if (!batch_state(B, offset, step, par)) return;
    const unsigned w = (unsigned)(blockIdx.x - pre[g]) * 8u + (threadIdx.x >> 5);
    if (w >= B.bh.wz + B.bh.wy + B.bh.wx) return;
    band_h_warp<float, false>(B.ph[par], B.bh, w, threadIdx.x & 31, step - B.probe_base, B.hout[par]);
}

__global__ void __launch_bounds__(256) band_e_batched(const BatchGrid *G, const int *pre, int n, int offset)
{
    const int g = find_slot(pre, n, blockIdx.x);
    const BatchGrid &B = G[g];
    long long step;
    int par;
    if (!batch_state(B, offset, step, par)) return;
    const unsigned w = (unsigned)(blockIdx.x - pre[g]) * 8u + (threadIdx.x >> 5);
    if (w >= B.be.wz + B.be.wy + B.be.wx) return;
    band_e_warp<float, false>(B.pe[par], B.be, w, threadIdx.x & 31, step, step - B.probe_base, B.eout[par]);
}

// ---------------------------------------------------------------------------
// Persistent batched step: one launch advances every grid of a batch by K
// steps.  CTAs take tickets from a counter in increasing order; ticket t is
// item t mod T of step t div T.  The T items of a step go grid by grid, and
// within a grid: its band-H items, its one-pass tiles, its band-E items (a
// band item is kBandGroup band CTAs' worth of warps).  An item of grid g at
// step o starts once every item of g at step o-1 has finished, a band-E item
// also once g's band-H items of step o have (per-grid counters,
// release/acquire).  A CTA only ever waits for items with smaller tickets,
// which CTAs already running hold, so the launch progresses however many of
// its CTAs are resident; with several grids a grid's next step is ready long
// before its ticket comes up, so grids at different steps overlap.  Every
// wait is bounded: on expiry the CTA raises the error flag, and every CTA
// stops taking work once the flag is up.
// ---------------------------------------------------------------------------
constexpr int kBandGroup = 8;

struct Persist {
    unsigned *ticket;        // ticket counter (zero at launch)
    unsigned *done;          // per grid g: [2g] items finished, [2g+1] band-H items finished (zero at launch)
    int *error_flag;         // raised when a wait gives up
    unsigned wait_limit;     // polls before a wait gives up
    int K;                   // steps in this launch
    int n;                   // grids
    int cap;                 // prefix table stride - 1
    int total;               // items per step, all grids
};

// Band items of a grid with `ctas` band CTAs.
__host__ __device__ __forceinline__ int band_items(int ctas) { return (ctas + kBandGroup - 1) / kBandGroup; }

// Items of grid g (band H, tiles, band E) from the three CTA prefix tables.
__device__ __forceinline__ void grid_items(const int *pf, const int *ph, const int *pe, int g, int &nh, int &nf,
                                           int &ne)
{
    nh = band_items(ph[g + 1] - ph[g]);
    nf = pf[g + 1] - pf[g];
    ne = band_items(pe[g + 1] - pe[g]);
}

// Wait (bounded) until *ctr >= target; false if the limit runs out or another
// CTA has already raised the error flag (then nothing further can complete).
__device__ __forceinline__ bool wait_count(const unsigned *ctr, unsigned target, unsigned limit, const int *error_flag)
{
    for (unsigned it = 0; it < limit; ++it) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) return true;
        if ((it & 255u) == 255u && *reinterpret_cast<const volatile int *>(error_flag)) return false;
        __nanosleep(it < 64 ? 32 : 256);
    }
    return false;
}

__global__ void __launch_bounds__(kFTY * 32, kStages <= 3 ? 3 : 2)
    persistent_batched(const BatchGrid *G, const int *pre, const int *pitems, const Persist P)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ unsigned s_ticket;
    __shared__ int s_go;
    const int *pf = pre, *ph = pre + (P.cap + 1), *pe = pre + 2 * (P.cap + 1);
    const unsigned end = (unsigned)P.K * (unsigned)P.total;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        // no new work once a wait has given up anywhere: every later item could
        // depend on the one that did not finish
        if (threadIdx.x == 0)
            s_ticket = *reinterpret_cast<const volatile int *>(P.error_flag) ? end : atomicAdd(P.ticket, 1u);
        __syncthreads();
        const unsigned t = s_ticket;
        if (t >= end) return;
        const int o = (int)(t / (unsigned)P.total);
        int r = (int)(t - (unsigned)o * (unsigned)P.total);
        const int g = find_slot(pitems, P.n, r);        // pitems: prefix of the grids' item counts
        r -= pitems[g];
        int nh, nf, ne;
        grid_items(pf, ph, pe, g, nh, nf, ne);
        const int kind = r < nh ? 0 : r < nh + nf ? 1 : 2;
        r -= kind == 0 ? 0 : kind == 1 ? nh : nh + nf;
        if (threadIdx.x == 0) {
            const unsigned items_g = (unsigned)(nh + nf + ne);
            bool ok = o == 0 || wait_count(&P.done[2 * g], (unsigned)o * items_g, P.wait_limit, P.error_flag);
            if (ok && kind == 2)
                ok = wait_count(&P.done[2 * g + 1], (unsigned)(o + 1) * (unsigned)nh, P.wait_limit, P.error_flag);
            if (!ok) atomicExch(P.error_flag, 1);
            // the tiles' TMA loads (async proxy) read what other CTAs stored
            asm volatile("fence.proxy.async.global;" ::: "memory");
            s_go = ok;
        }
        __syncthreads();
        if (!s_go) return;
        const BatchGrid &B = G[g];
        long long step;
        int par;
        if (batch_state(B, o, step, par)) {
            if (kind == 1) {
                const int tx = B.tiles[0], ty = B.tiles[1];
                fused_body<true, float>(B.maps[par], B.fp[par], step, step - B.probe_base, r % tx, (r / tx) % ty,
                                        r / (tx * ty), smem_raw);
            } else if (kind == 0) {
                const unsigned nw = B.bh.wz + B.bh.wy + B.bh.wx;
                for (unsigned w = (unsigned)r * (8u * kBandGroup) + (unsigned)warp;
                     w < nw && w < (unsigned)(r + 1) * (8u * kBandGroup); w += 8u)
                    band_h_warp<float, false, true>(B.ph[par], B.bh, w, lane, step - B.probe_base, B.hout[par]);
            } else {
                const unsigned nw = B.be.wz + B.be.wy + B.be.wx;
                for (unsigned w = (unsigned)r * (8u * kBandGroup) + (unsigned)warp;
                     w < nw && w < (unsigned)(r + 1) * (8u * kBandGroup); w += 8u)
                    band_e_warp<float, false, true>(B.pe[par], B.be, w, lane, step, step - B.probe_base,
                                                    B.eout[par]);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (kind == 0) atomicAdd(&P.done[2 * g + 1], 1u);
            atomicAdd(&P.done[2 * g], 1u);
        }
    }
}

__global__ void batch_advance(const BatchGrid *G, int n, long long k)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const long long c = *G[g].counter, t = G[g].target;
    *G[g].counter = c + k < t ? c + k : (c < t ? t : c);
}

}  // namespace sbp
