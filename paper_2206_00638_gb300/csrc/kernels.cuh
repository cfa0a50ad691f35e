// Device code of the GB300 SBP-SAT FDTD library (arXiv 2206.00638).
//
// Two fused kernels advance one leapfrog step:
//   h_update  H^{n+1/2} = H^{n-1/2} + dt/mu (D- E^n) + SAT_H     Eqs. (10)-(15), Alg. 2
//   e_update  E^{n+1}   = E^n + dt/eps (D+ H^{n+1/2} - J) + SAT_E Eqs. (7)-(9), (19)-(21), Alg. 1
// Each thread owns one (i, j) column of nodes and marches up a chunk of z
// planes (2.5D blocking): the z-neighbour needed by the staggered difference
// is carried in a register from the previous plane, x/y neighbours come from
// L1.  Interior nodes (every index in [3, n-2]) take a branch-free fast path
// with the two-point stencil; the three boundary layers of each axis take the
// general path, which evaluates the closure rows of D+ / D- (Appendix), the
// SAT penalties of the face type (PEC / PMC / absorbing / interface), point
// and sheet sources and probes.  The fast/general choice is uniform per warp
// except in the two x-edge warps of a row.
//
// FP32 arithmetic keeps its coefficients exact to ~1e-14: every material
// coefficient dt/(eps h) is carried as an unevaluated sum hi + lo of two
// floats, and the node's 1/sum(eps_r) as a Newton-corrected reciprocal pair,
// so rounding of a coefficient does not bias the phase velocity; only the
// per-step rounding of the field update (unbiased) remains.
#pragma once
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

namespace sbp {

constexpr int kMaxSources = 16;
constexpr int kMaxProbes = 64;
constexpr int kBlockX = 32;
constexpr int kBlockY = 8;

enum : int { kPEC = 0, kPMC = 1, kABS = 2, kIFACE = 3 };

// Table I: component c lives on the plus grid (n+1 nodes) along axis a.
__host__ __device__ constexpr bool on_plus(int c, int a)
{
    return c == 0 ? a != 0 : c == 1 ? a != 1 : c == 2 ? a != 2
         : c == 3 ? a == 0 : c == 4 ? a == 1 : a == 2;
}

// Eqs. (7)-(12): dC/dt = (+1) D^{axis0} C0 + (-1) D^{axis1} C1.
__host__ __device__ constexpr int curl_comp(int c, int t)
{
    // Ex: Hz, Hy   Ey: Hx, Hz   Ez: Hy, Hx   Hx: Ey, Ez   Hy: Ez, Ex   Hz: Ex, Ey
    return t == 0 ? (c == 0 ? 5 : c == 1 ? 3 : c == 2 ? 4 : c == 3 ? 1 : c == 4 ? 2 : 0)
                  : (c == 0 ? 4 : c == 1 ? 5 : c == 2 ? 3 : c == 3 ? 2 : c == 4 ? 0 : 1);
}
__host__ __device__ constexpr int curl_axis(int c, int t)
{
    // Ex: y, z   Ey: z, x   Ez: x, y   Hx: z, y   Hy: x, z   Hz: y, x
    return t == 0 ? (c == 0 ? 1 : c == 1 ? 2 : c == 2 ? 0 : c == 3 ? 2 : c == 4 ? 0 : 1)
                  : (c == 0 ? 2 : c == 1 ? 0 : c == 2 ? 1 : c == 3 ? 1 : c == 4 ? 2 : 0);
}
__host__ __device__ constexpr int curl_sign(int t) { return t == 0 ? 1 : -1; }

template <typename T> struct Coef { T hi, lo; };

struct Link {               // interface partner of one face
    const void *F[6];       // partner block's padded fields
    const void *G[6];       // second partner (phase-shifted periodic face of a complex pair), or null
    double w[2];            // partner value = w[0] F + w[1] G (used when G is set)
    long long sy, sz;       // partner strides (elements)
    int n_norm;             // partner cell count along the face normal
    int side;               // partner face side: -1 low, +1 high
};

struct Src { int comp, i, j, k, wf; double amp, tw, t0, f; };
struct Prb { int comp, i, j, k; };

// Field storage type S and the arithmetic type of its values: FP16 storage
// is computed in FP32.
template <typename S> struct Compute { using type = S; };
template <> struct Compute<__half> { using type = float; };
template <typename S> using compute_t = typename Compute<S>::type;

// T: arithmetic type; S: storage type of the six fields (T, or __half with
// T = float).  Stored FP16 values are field / scale, one scale for E and one
// for H; the curl coefficients below carry the ratio of the two scales, so a
// kernel only converts on load and store.
template <typename T, typename S = T>
struct Params {
    S *F[6];                // padded fields Ex..Hz: element (i,j,k) at k*sz + j*sy + i
    const float *eps;       // ghost-padded cell eps_r on the same layout: cell (cx,cy,cz) at (cx+1,cy+1,cz+1)
    const float *mu;        // same for mu_r (only read when MUVAR)
    int n[3];
    long long sy, sz;
    int face[6];
    Link link[6];
    Coef<T> B[3];           // H: dt/(mu0 h_a) (uniform mu) or 2 dt/(mu0 h_a) (scaled by 1/sum2 mu_r)
    Coef<T> A[3];           // E: 4 dt/(eps0 h_a), scaled by 1/sum4 eps_r of the node
    Coef<T> AJ;             // 4 dt/eps0, source term
    double dt, eta0, eps0, mu0;
    double h[3];
    int nsrc, nprb;
    Src src[kMaxSources];
    Prb prb[kMaxProbes];
    T fscale[2];                       // physical value = stored value * fscale[E=0 / H=1]
    T uB, uA;                          // fscale[H]/fscale[E] and its inverse: B and A carry the
                                       // scale ratio; the absorbing-SAT gamma needs them without
    T *probe_buf;
    long long probe_cap, probe_slot;   // sample slot of this step (skip if >= cap)
    long long step;                    // n: the E half-step injects J(t^{n+1/2})
    double *partials;                  // energy partial sums, one per CTA of h_update
    int kchunk;
    int fdtd;                          // 1: plain Yee FDTD comparator (band kernels only)
};

// ---------------------------------------------------------------------------
// small arithmetic helpers
// ---------------------------------------------------------------------------
template <typename T> struct Acc;
template <> struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(const Coef<float> &c, float x, float scale = 1.f)
    {
        hi = fmaf(scale * c.hi, x, hi);
        lo = fmaf(scale * c.lo, x, lo);
    }
};
template <> struct Acc<double> {
    double hi = 0.0;
    __device__ __forceinline__ void add(const Coef<double> &c, double x, double scale = 1.0)
    {
        hi = fma(scale * c.hi, x, hi);
    }
};

// Reciprocal of s as hi + lo (hardware approximation + one Newton residual).
__device__ __forceinline__ void recip_pair(float s, float &rh, float &rl)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
    float e = fmaf(-s, r, 1.0f);
    rh = r;
    rl = r * e;
}

// increment = r * acc with r = 1/s (E nodes, or H nodes with varying mu)
__device__ __forceinline__ float scaled_increment(const Acc<float> &a, float s)
{
    float rh, rl;
    recip_pair(s, rh, rl);
    return fmaf(rh, a.hi, fmaf(rh, a.lo, rl * a.hi));
}
__device__ __forceinline__ double scaled_increment(const Acc<double> &a, double s)
{
    return a.hi / s;
}
__device__ __forceinline__ float plain_increment(const Acc<float> &a) { return a.hi + a.lo; }
__device__ __forceinline__ double plain_increment(const Acc<double> &a) { return a.hi; }

// FP32 arithmetic on FP16-stored fields: the coefficients' rounding residue
// (lo, about 6e-8 relative) is far below the storage rounding (4.9e-4), so
// the increment is accumulated from the rounded coefficients alone.
struct AccLite {
    float hi = 0.f;
    __device__ __forceinline__ void add(const Coef<float> &c, float x, float scale = 1.f)
    {
        hi = fmaf(scale * c.hi, x, hi);
    }
};
__device__ __forceinline__ float scaled_increment(const AccLite &a, float s)
{
    float rh, rl;
    recip_pair(s, rh, rl);
    return fmaf(rh, a.hi, rl * a.hi);
}
__device__ __forceinline__ float plain_increment(const AccLite &a) { return a.hi; }

// The accumulator of arithmetic type T for fields stored as S.
template <typename T, typename S> struct AccOf { using type = Acc<T>; };
template <> struct AccOf<float, __half> { using type = AccLite; };

// Rows of the Appendix operators at unit spacing.  Every row reads at most
// three consecutive entries of its line; they are gathered first (no branch
// before the loads, so all of a node's loads are in flight together) and the
// row formula is then applied to them.  The line holds entries 0..n+1 of the
// padded layout, so the gathered triple is always in bounds.
template <typename T> struct Tri { T a, b, c; };

// Field loads and stores in the storage type, values in the arithmetic type.
template <typename S>
__device__ __forceinline__ compute_t<S> ld_s(const S *p)
{
    if constexpr (std::is_same<S, __half>::value) return __half2float(*p);
    else return *p;
}
template <typename S>
__device__ __forceinline__ compute_t<S> ldg_s(const S *p)
{
    if constexpr (std::is_same<S, __half>::value) return __half2float(__ldg(p));
    else return __ldg(p);
}
// CG = true reads through L2 only (ld.global.cg), for values this kernel
// itself wrote earlier (coherent across the threads of a CTA after a
// barrier, never served stale from L1 or the read-only path).
template <bool CG, typename S>
__device__ __forceinline__ compute_t<S> ldf(const S *p)
{
    if constexpr (CG) {
        if constexpr (std::is_same<S, __half>::value) return __half2float(__ldcg(p));
        else return __ldcg(p);
    } else {
        return ld_s(p);
    }
}
// The value a store of v keeps (round to nearest for FP16 storage).
template <typename S, typename T>
__device__ __forceinline__ T quant(T v)
{
    if constexpr (std::is_same<S, __half>::value) return __half2float(__float2half_rn(v));
    else return v;
}
template <typename S, typename T>
__device__ __forceinline__ void st_s(S *p, T v)
{
    if constexpr (std::is_same<S, __half>::value) *p = __float2half_rn(v);
    else *p = v;
}

// entries s0, s0+1, s0+2 of the line starting at `line` with stride s
template <bool CG, typename S>
__device__ __forceinline__ Tri<compute_t<S>> tri_load(const S *line, long long s, int s0)
{
    const S *q = line + (long long)s0 * s;
    return {ldf<CG>(q), ldf<CG>(q + s), ldf<CG>(q + 2 * s)};
}

// FMA in the arithmetic type.
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// A row of either operator reads at most three consecutive entries u_a, u_b,
// u_c of its line, with coefficients k0, k1, k2 (unit spacing).  Every kernel
// evaluates a row as the same chain, entries in increasing index order:
//   d = k0 u_a;  d = fma(k1, u_b, d);  d = fma(k2, u_c, d).
// A zero coefficient leaves d unchanged, and an interior row (-1, 1, 0)
// gives u_b - u_a exactly as a subtraction does, so the interior fast paths
// (plain differences), the one-pass kernel's x-end windows (four entries,
// zeros outside the row) and the general path all produce the same bits.
template <typename T>
__device__ __forceinline__ T row_chain(const T k[3], T a, T b, T c)
{
    T d = k[0] * a;
    d = fma_t(k[1], b, d);
    return fma_t(k[2], c, d);
}

// D- : x+ (n+1 values) -> x- (n+2 rows).  First entry read by row r.
__device__ __forceinline__ int dminus_start(int r, int n)
{
    return (r == 0 || r == 2) ? 0 : (r == n - 1 || r == n + 1) ? n - 2 : r - 1;
}
// Coefficients of row r of D- on the entries at dminus_start(r, n) (Appendix).
template <typename T>
__device__ __forceinline__ void dminus_coefs(int r, int n, T k[3])
{
    if (r == 2) { k[0] = T(-0.2); k[1] = T(-0.6); k[2] = T(0.8); }              // (4u2 - 3u1 - u0) / 5
    else if (r == n - 1) { k[0] = T(-0.8); k[1] = T(0.6); k[2] = T(0.2); }      // (u_n + 3u_{n-1} - 4u_{n-2}) / 5
    else if (r == n + 1) { k[0] = T(0); k[1] = T(-1); k[2] = T(1); }            // u_n - u_{n-1}
    else { k[0] = T(-1); k[1] = T(1); k[2] = T(0); }                            // rows 0 (u1 - u0), 1, 3..n-2, n
}
// Row r of D- from the entries gathered at dminus_start(r, n).
template <typename T>
__device__ __forceinline__ T dminus_eval(const Tri<T> &u, int r, int n)
{
    T k[3];
    dminus_coefs(r, n, k);
    return row_chain(k, u.a, u.b, u.c);
}

// D+ : x- (n+2 values) -> x+ (n+1 rows).  First entry read by row r.
__device__ __forceinline__ int dplus_start(int r, int n) { return r <= 1 ? 0 : r >= n - 1 ? n - 1 : r; }
// Coefficients of row r of D+ on the entries at dplus_start(r, n) (Appendix).
template <typename T>
__device__ __forceinline__ void dplus_coefs(int r, int n, T k[3])
{
    if (r == 0) { k[0] = T(-1); k[1] = T(0.5); k[2] = T(0.5); }                 // (v1 + v2)/2 - v0
    else if (r == 1) { k[0] = T(-0.5); k[1] = T(-0.25); k[2] = T(0.75); }       // 3v2/4 - v0/2 - v1/4
    else if (r == n - 1) { k[0] = T(-0.75); k[1] = T(0.25); k[2] = T(0.5); }    // v_n/4 + v_{n+1}/2 - 3v_{n-1}/4
    else if (r == n) { k[0] = T(-0.5); k[1] = T(-0.5); k[2] = T(1); }           // v_{n+1} - (v_{n-1} + v_n)/2
    else { k[0] = T(-1); k[1] = T(1); k[2] = T(0); }                            // rows 2..n-2: v_{r+1} - v_r
}
// Row r of D+ from the entries gathered at dplus_start(r, n).
template <typename T>
__device__ __forceinline__ T dplus_eval(const Tri<T> &v, int r, int n)
{
    T k[3];
    dplus_coefs(r, n, k);
    return row_chain(k, v.a, v.b, v.c);
}

// SAT helpers shared by every kernel that evaluates a face node, so that all
// of them round alike.
// Penalty value of an interface face: the partner's field at its face node,
// or e^{-+j alpha} times the complex partner (real and imaginary simulations).
template <bool CG, typename T, typename S>
__device__ __forceinline__ T link_value(const Link &L, int u, long long on)
{
    T nv = ldf<CG>(static_cast<const S *>(L.F[u]) + on);
    if (L.G[u]) nv = fma_t(T(L.w[1]), T(ldf<CG>(static_cast<const S *>(L.G[u]) + on)), T(L.w[0]) * nv);
    return nv;
}
// Characteristic impedance eta0 sqrt(mu_r / eps_r) at the node.
template <typename T>
__device__ __forceinline__ T node_eta(double eta0, T mr, T er) { return T(eta0) * sqrt(mr / er); }
// Absorbing penalty, H side: gamma = dt eta / (2 mu h) = (1/2) ba eta, ba = dt / (mu h) in stored units.
template <typename T>
__device__ __forceinline__ T abs_gamma_h(T ba, T eta) { return T(0.5) * ba * eta; }
// Absorbing penalty, E side: gamma = dt / (2 eta eps h) = (a / se) / (2 eta), a = 4 dt / (eps0 h) in
// stored units and se = 4 eps_r of the node.
template <typename T>
__device__ __forceinline__ T abs_gamma_e(T a, T se, T eta) { return a / se / (T(2) * eta); }
// New value with the absorbing self term averaged over the two time levels
// (pointwise semi-implicit): ((1 - gamma) old + inc) / (1 + gamma).
template <typename T>
__device__ __forceinline__ T sat_finish(T old, T inc, T gam)
{
    if (gam != T(0)) return fma_t(T(1) - gam, old, inc) / (T(1) + gam);
    return old + inc;
}

// 1D norm weight (unit spacing) of node r: P+ = diag(1/2,1,...,1,1/2),
// P- = diag(1/2,1/4,5/4,1,...,1,5/4,1/4,1/2)  (Appendix).
__device__ __forceinline__ double norm_weight(bool plus, int r, int n)
{
    if (plus) return (r == 0 || r == n) ? 0.5 : 1.0;
    if (r == 0 || r == n + 1) return 0.5;
    if (r == 1 || r == n) return 0.25;
    if (r == 2 || r == n - 1) return 1.25;
    return 1.0;
}

__device__ __forceinline__ int extent(const int n[3], int c, int a) { return n[a] + (on_plus(c, a) ? 1 : 2); }

// (m[o] + m[o+a]) + (m[o+b] + m[o+a+b])
template <typename S>
__device__ __forceinline__ S pair_sum(const float *__restrict__ m, long long o, long long a, long long b)
{
    return (S(__ldg(m + o)) + S(__ldg(m + o + a))) + (S(__ldg(m + o + b)) + S(__ldg(m + o + a + b)));
}

// Sum of the ghost-padded cell values around a node of component c: the
// closed-box cell set of the node, always 2x2 (E) or 2x1 (H) entries after
// ghost padding (duplicates stand for clipped cells, so the mean is the mean
// over the distinct cells).
template <int C, typename S = float>
__device__ __forceinline__ S cell_sum(const float *__restrict__ m, long long o, long long sy, long long sz)
{
    // ghost-padded index of the node's first cell is the node index itself;
    // a plus-grid axis spans two cells (offset 0 and +1), a minus-grid axis one.
    // Summed pairwise, (a + b) + (c + d): exact whenever the cells agree, and
    // the same order in the fast and the general path.
    constexpr bool px = on_plus(C, 0), py = on_plus(C, 1), pz = on_plus(C, 2);
    if (px && py) return pair_sum<S>(m, o, 1, sy);
    if (px && pz) return pair_sum<S>(m, o, 1, sz);
    if (py && pz) return pair_sum<S>(m, o, sy, sz);
    const long long d = px ? 1 : py ? sy : sz;
    return S(__ldg(m + o)) + S(__ldg(m + o + d));
}
// number of entries summed by cell_sum<C>
__host__ __device__ constexpr int cell_count(int c)
{
    return (on_plus(c, 0) ? 2 : 1) * (on_plus(c, 1) ? 2 : 1) * (on_plus(c, 2) ? 2 : 1);
}

// Source waveforms (Sec. VI-B, VI-C): t and t0, tw in seconds.
__device__ __forceinline__ double waveform(int wf, double t, double tw, double t0, double f)
{
    const double x = (t - t0) / tw;
    const double g = exp(-4.0 * 3.14159265358979323846 * x * x);
    if (wf == 0) return g;
    if (wf == 1) return -5.0132565492620005 * x * 1.6487212707001282 * g;   // -sqrt(8 pi) x e^{1/2} g
    double ph = f * t;
    ph -= floor(ph);
    return sin(6.283185307179586 * ph) * g;
}

template <typename T, typename S>
__device__ __forceinline__ bool probe_here(const Params<T, S> &p, unsigned long long mask, int k)
{
    while (mask) {
        int q = __ffsll(mask) - 1;
        mask &= mask - 1;
        if (p.prb[q].k == k) return true;
    }
    return false;
}
template <typename T, typename S>
__device__ __forceinline__ bool source_here(const Params<T, S> &p, unsigned mask, int k)
{
    while (mask) {
        int q = __ffs(mask) - 1;
        mask &= mask - 1;
        if (p.src[q].k == k || p.src[q].k < 0) return true;
    }
    return false;
}
template <typename T, typename S>
__device__ __forceinline__ void write_probes(const Params<T, S> &p, unsigned long long mask, int c, int k, T v)
{
    while (mask) {
        int q = __ffsll(mask) - 1;
        mask &= mask - 1;
        if (p.prb[q].comp == c && p.prb[q].k == k && p.probe_slot < p.probe_cap)
            p.probe_buf[(long long)q * p.probe_cap + p.probe_slot] = v * p.fscale[c >= 3];
    }
}

// Block-wide deterministic sum of one double per thread (fixed tree).
__device__ __forceinline__ void block_sum_to(double v, double *dst)
{
    __shared__ double red[kBlockX * kBlockY / 32];
    const int lane = threadIdx.x, warp = threadIdx.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)blockDim.y ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) *dst = v;
    }
}

// ---------------------------------------------------------------------------
// H half-step: general path for one component at one node
// ---------------------------------------------------------------------------
// Entries of E read by the two curl terms of H component C at node idx.
// G: bit a set when the node may lie on a closure row or face along axis a;
// along the other axes the node is interior and the row is u_r - u_{r-1}.
// CG: read through L2 only (fields another CTA of the same launch wrote).
template <typename T, int C, int G = 7, bool CG = false, typename S = T>
__device__ __forceinline__ void h_gather(const Params<T, S> &p, const int idx[3], long long o, Tri<T> v[2])
{
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int u = curl_comp(C, t), a = curl_axis(C, t);
        const long long st = a == 0 ? 1 : a == 1 ? p.sy : p.sz;
        if ((G >> a) & 1) {
            v[t] = tri_load<CG>(p.F[u] + (o - idx[a] * st), st, dminus_start(idx[a], p.n[a]));
        } else {
            v[t].a = ldf<CG>(p.F[u] + o - st);
            v[t].b = ldf<CG>(p.F[u] + o);
            v[t].c = v[t].b;
        }
    }
}

// H^{n+1/2} of component C at node idx from H^{n-1/2} (hold) and the gathered E.
template <typename T, int C, bool MUVAR, int G = 7, typename S = T>
__device__ __forceinline__ T h_apply(const Params<T, S> &p, const int idx[3], long long o, T hold, const Tri<T> v[2])
{
    typename AccOf<T, S>::type acc;
    T gam = T(0);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int u = curl_comp(C, t), a = curl_axis(C, t), sg = curl_sign(t);
        const bool gen = (G >> a) & 1;
        const T d = gen ? dminus_eval(v[t], idx[a], p.n[a]) : v[t].b - v[t].a;
        acc.add(p.B[a], d, T(sg));
        // H on the minus grid along a: face nodes at 0 and n+1 carry the SAT
        if (gen && (idx[a] == 0 || idx[a] == p.n[a] + 1)) {
            const int side = idx[a] == 0 ? -1 : 1;
            const int f = 2 * a + (side > 0);
            const int type = p.face[f];
            if (type != kPMC) {
                const T phi = T(-sg * side);
                const T pv = side < 0 ? v[t].a : v[t].c;      // E on the face: entry 0 or n
                if (type == kPEC) {
                    acc.add(p.B[a], pv, T(2) * phi);
                } else if (type == kABS) {
                    acc.add(p.B[a], pv, phi);
                    const T er = cell_sum<C, T>(p.eps, o, p.sy, p.sz) * T(0.5);
                    const T mr = MUVAR ? cell_sum<C, T>(p.mu, o, p.sy, p.sz) * T(0.5) : T(1);
                    // B holds dt/(mu0 h_a) (x2 when mu varies)
                    const T ba = (MUVAR ? T(p.B[a].hi) * T(0.5) / mr : T(p.B[a].hi)) * p.uB;
                    gam += abs_gamma_h(ba, node_eta(p.eta0, mr, er));
                } else {   // interface: (phi/2)(E^A - E^B) / (mu w), w = h/2
                    const Link &L = p.link[f];
                    const int nidx = L.side < 0 ? 0 : L.n_norm;      // partner E on its plus grid along a
                    long long on = 0;
                    const long long ost[3] = {1, L.sy, L.sz};
                    for (int b = 0; b < 3; ++b) on += (long long)(b == a ? nidx : idx[b]) * ost[b];
                    acc.add(p.B[a], pv - link_value<false, T, S>(L, u, on), phi);
                }
            }
        }
    }
    T inc;
    if (MUVAR) {
        inc = scaled_increment(acc, cell_sum<C, T>(p.mu, o, p.sy, p.sz));
    } else {
        inc = plain_increment(acc);
    }
    return sat_finish(hold, inc, gam);
}

// H half-step, general path, one component at one node (Eqs. (10)-(15)).
template <typename T, int C, bool MUVAR, typename S = T>
__device__ __forceinline__ T h_node(const Params<T, S> &p, const int idx[3], long long o, T hold)
{
    Tri<T> v[2];
    h_gather<T, C, 7>(p, idx, o, v);
    return h_apply<T, C, MUVAR, 7>(p, idx, o, hold, v);
}

// Entries of H read by the two curl terms of E component C at node idx.
// G as for h_gather; interior rows of D+ are v_{r+1} - v_r.
template <typename T, int C, bool CG = false, int G = 7, typename S = T>
__device__ __forceinline__ void e_gather(const Params<T, S> &p, const int idx[3], long long o, Tri<T> v[2])
{
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int u = curl_comp(C, t), a = curl_axis(C, t);
        const long long st = a == 0 ? 1 : a == 1 ? p.sy : p.sz;
        if ((G >> a) & 1) {
            v[t] = tri_load<CG>(p.F[u] + (o - idx[a] * st), st, dplus_start(idx[a], p.n[a]));
        } else {
            v[t].a = ldf<CG>(p.F[u] + o);
            v[t].b = ldf<CG>(p.F[u] + o + st);
            v[t].c = v[t].b;
        }
    }
}

// E^{n+1} of component C at node idx from E^n (eold), se = sum4 eps_r of the
// node and the gathered H.
template <typename T, int C, bool MUVAR, bool CG = false, int G = 7, typename S = T>
__device__ __forceinline__ T e_apply(const Params<T, S> &p, const int idx[3], long long o, T eold, T se, const Tri<T> v[2],
                                     unsigned smask, double t_half)
{
    typename AccOf<T, S>::type acc;
    T gam = T(0);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int u = curl_comp(C, t), a = curl_axis(C, t), sg = curl_sign(t);
        const bool gen = (G >> a) & 1;
        const T d = gen ? dplus_eval(v[t], idx[a], p.n[a]) : v[t].b - v[t].a;
        acc.add(p.A[a], d, T(sg));
        // E on the plus grid along a: face nodes at 0 and n carry the SAT
        if (gen && (idx[a] == 0 || idx[a] == p.n[a])) {
            const int side = idx[a] == 0 ? -1 : 1;
            const int f = 2 * a + (side > 0);
            const int type = p.face[f];
            if (type != kPEC) {
                const T phi = T(-sg * side);
                const T pv = side < 0 ? v[t].a : v[t].c;      // H on the face: entry 0 or n+1
                if (type == kPMC) {
                    acc.add(p.A[a], pv, T(2) * phi);
                } else if (type == kABS) {
                    acc.add(p.A[a], pv, phi);
                    const T er = se * T(0.25);
                    const T mr = MUVAR ? cell_sum<C, T>(p.mu, o, p.sy, p.sz) * T(0.25) : T(1);
                    gam += abs_gamma_e(T(p.A[a].hi) * p.uA, se, node_eta(p.eta0, mr, er));
                } else {
                    const Link &L = p.link[f];
                    const int nidx = L.side < 0 ? 0 : L.n_norm + 1;  // partner H on its minus grid along a
                    long long on = 0;
                    const long long ost[3] = {1, L.sy, L.sz};
                    for (int b = 0; b < 3; ++b) on += (long long)(b == a ? nidx : idx[b]) * ost[b];
                    acc.add(p.A[a], pv - link_value<CG, T, S>(L, u, on), phi);
                }
            }
        }
    }
    // current-density sources: eps dE/dt = ... - J
    unsigned m = smask;
    while (m) {
        const int q = __ffs(m) - 1;
        m &= m - 1;
        const Src &Sr = p.src[q];
        if (Sr.comp == C && (Sr.k < 0 || Sr.k == idx[2])) {
            const double J = Sr.amp * waveform(Sr.wf, t_half, Sr.tw, Sr.t0, Sr.f);
            acc.add(p.AJ, T(J), T(-1));
        }
    }
    const T inc = scaled_increment(acc, se);
    return sat_finish(eold, inc, gam);
}

// E half-step, general path, one component at one node (Eqs. (7)-(9), (19)-(21)).
template <typename T, int C, bool MUVAR, bool CG = false, typename S = T>
__device__ __forceinline__ T e_node(const Params<T, S> &p, const int idx[3], long long o, T eold,
                                    unsigned smask, double t_half)
{
    const T se = cell_sum<C, T>(p.eps, o, p.sy, p.sz);     // 4 * eps_r(node)
    Tri<T> v[2];
    e_gather<T, C, CG, 7>(p, idx, o, v);
    return e_apply<T, C, MUVAR, CG, 7>(p, idx, o, eold, se, v, smask, t_half);
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Per-thread masks of the probes / sources whose (i, j) match this column.
template <typename T, typename S>
__device__ __forceinline__ void column_masks(const Params<T, S> &p, int i, int j, bool want_h,
                                             unsigned long long &pm, unsigned &sm)
{
    pm = 0ull;
    sm = 0u;
    for (int q = 0; q < p.nprb; ++q)
        if (p.prb[q].i == i && p.prb[q].j == j && ((p.prb[q].comp >= 3) == want_h)) pm |= 1ull << q;
    if (!want_h)
        for (int q = 0; q < p.nsrc; ++q)
            if ((p.src[q].i < 0 || p.src[q].i == i) && (p.src[q].j < 0 || p.src[q].j == j)) sm |= 1u << q;
}

// H half-step.  ENERGY: also accumulate the leapfrog energy of Eq. (16) into
// p.partials (FP64); STORE: write H^{n+1/2} (false = energy query only).
template <typename T, typename S, bool ENERGY, bool STORE, bool MUVAR>
__global__ void __launch_bounds__(kBlockX *kBlockY) h_update(const Params<T, S> p)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    const int k0 = blockIdx.z * p.kchunk;
    const int k1 = min(k0 + p.kchunk, nz + 2);
    double wacc = 0.0;
    if (i < nx + 2 && j < ny + 2) {
        S *__restrict__ Hx = p.F[3];
        S *__restrict__ Hy = p.F[4];
        S *__restrict__ Hz = p.F[5];
        const S *__restrict__ Ex = p.F[0];
        const S *__restrict__ Ey = p.F[1];
        const S *__restrict__ Ez = p.F[2];
        const double es2 = (double)p.fscale[0] * (double)p.fscale[0];   // energy of stored values
        const double hs2 = (double)p.fscale[1] * (double)p.fscale[1];
        unsigned long long pm;
        unsigned sm;
        column_masks(p, i, j, true, pm, sm);
        const bool xyin = i >= 3 && i <= nx - 2 && j >= 3 && j <= ny - 2;
        const Coef<T> Bx = p.B[0], By = p.B[1], Bz = p.B[2];
        long long o = (long long)k0 * p.sz + (long long)j * p.sy + i;
        T exm = k0 > 0 ? ldg_s(Ex + o - p.sz) : T(0);
        T eym = k0 > 0 ? ldg_s(Ey + o - p.sz) : T(0);
        for (int k = k0; k < k1; ++k, o += p.sz) {
            const T exc = ldg_s(Ex + o);
            const T eyc = ldg_s(Ey + o);
            const bool fast = !ENERGY && !MUVAR && xyin && k >= 3 && k <= nz - 2 && !(pm && probe_here(p, pm, k));
            if (fast) {
                const T ezc = ldg_s(Ez + o);
                const T ex_jm = ldg_s(Ex + o - p.sy);
                const T ey_im = ldg_s(Ey + o - 1);
                const T ez_im = ldg_s(Ez + o - 1);
                const T ez_jm = ldg_s(Ez + o - p.sy);
                const T dEy_z = eyc - eym, dEz_y = ezc - ez_jm;
                const T dEz_x = ezc - ez_im, dEx_z = exc - exm;
                const T dEx_y = exc - ex_jm, dEy_x = eyc - ey_im;
                typename AccOf<T, S>::type ax, ay, az;
                ax.add(Bz, dEy_z); ax.add(By, dEz_y, T(-1));
                ay.add(Bx, dEz_x); ay.add(Bz, dEx_z, T(-1));
                az.add(By, dEx_y); az.add(Bx, dEy_x, T(-1));
                st_s(Hx + o, ld_s(Hx + o) + plain_increment(ax));
                st_s(Hy + o, ld_s(Hy + o) + plain_increment(ay));
                st_s(Hz + o, ld_s(Hz + o) + plain_increment(az));
            } else {
                const int idx[3] = {i, j, k};
                // Hx (x+, y-, z-)
                if (i <= nx && j <= ny + 1 && k <= nz + 1) {
                    const T ho = ld_s(Hx + o);
                    const T hn = quant<S>(h_node<T, 3, MUVAR>(p, idx, o, ho));
                    if (STORE) st_s(Hx + o, hn);
                    if (STORE && pm) write_probes(p, pm, 3, k, hn);
                    if (ENERGY) {
                        const double w = norm_weight(true, i, nx) * norm_weight(false, j, ny) * norm_weight(false, k, nz);
                        const double mr = MUVAR ? 0.5 * cell_sum<3, double>(p.mu, o, p.sy, p.sz) : 1.0;
                        wacc += p.mu0 * mr * w * (double)ho * (double)hn * hs2;
                    }
                }
                // Hy (x-, y+, z-)
                if (i <= nx + 1 && j <= ny && k <= nz + 1) {
                    const T ho = ld_s(Hy + o);
                    const T hn = quant<S>(h_node<T, 4, MUVAR>(p, idx, o, ho));
                    if (STORE) st_s(Hy + o, hn);
                    if (STORE && pm) write_probes(p, pm, 4, k, hn);
                    if (ENERGY) {
                        const double w = norm_weight(false, i, nx) * norm_weight(true, j, ny) * norm_weight(false, k, nz);
                        const double mr = MUVAR ? 0.5 * cell_sum<4, double>(p.mu, o, p.sy, p.sz) : 1.0;
                        wacc += p.mu0 * mr * w * (double)ho * (double)hn * hs2;
                    }
                }
                // Hz (x-, y-, z+)
                if (i <= nx + 1 && j <= ny + 1 && k <= nz) {
                    const T ho = ld_s(Hz + o);
                    const T hn = quant<S>(h_node<T, 5, MUVAR>(p, idx, o, ho));
                    if (STORE) st_s(Hz + o, hn);
                    if (STORE && pm) write_probes(p, pm, 5, k, hn);
                    if (ENERGY) {
                        const double w = norm_weight(false, i, nx) * norm_weight(false, j, ny) * norm_weight(true, k, nz);
                        const double mr = MUVAR ? 0.5 * cell_sum<5, double>(p.mu, o, p.sy, p.sz) : 1.0;
                        wacc += p.mu0 * mr * w * (double)ho * (double)hn * hs2;
                    }
                }
                if (ENERGY) {
                    // E^n part: eps P''' E^2 at this node position for every E component present
                    if (i <= nx + 1 && j <= ny && k <= nz) {   // Ex (x-, y+, z+)
                        const double w = norm_weight(false, i, nx) * norm_weight(true, j, ny) * norm_weight(true, k, nz);
                        wacc += p.eps0 * 0.25 * cell_sum<0, double>(p.eps, o, p.sy, p.sz) * w * (double)exc * (double)exc * es2;
                    }
                    if (i <= nx && j <= ny + 1 && k <= nz) {   // Ey (x+, y-, z+)
                        const double w = norm_weight(true, i, nx) * norm_weight(false, j, ny) * norm_weight(true, k, nz);
                        wacc += p.eps0 * 0.25 * cell_sum<1, double>(p.eps, o, p.sy, p.sz) * w * (double)eyc * (double)eyc * es2;
                    }
                    if (i <= nx && j <= ny && k <= nz + 1) {   // Ez (x+, y+, z-)
                        const double w = norm_weight(true, i, nx) * norm_weight(true, j, ny) * norm_weight(false, k, nz);
                        const T ezc = ldg_s(Ez + o);
                        wacc += p.eps0 * 0.25 * cell_sum<2, double>(p.eps, o, p.sy, p.sz) * w * (double)ezc * (double)ezc * es2;
                    }
                }
            }
            exm = exc;
            eym = eyc;
        }
    }
    if (ENERGY) {
        const double hvol = p.h[0] * p.h[1] * p.h[2];
        block_sum_to(wacc * hvol, p.partials + ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
    }
}

// E half-step with sources (J at t^{n+1/2}) and E probes.
template <typename T, typename S, bool MUVAR>
__global__ void __launch_bounds__(kBlockX *kBlockY) e_update(const Params<T, S> p)
{
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
    const int k0 = blockIdx.z * p.kchunk;
    const int k1 = min(k0 + p.kchunk, nz + 2);
    if (i >= nx + 2 || j >= ny + 2) return;
    S *__restrict__ Ex = p.F[0];
    S *__restrict__ Ey = p.F[1];
    S *__restrict__ Ez = p.F[2];
    const S *__restrict__ Hx = p.F[3];
    const S *__restrict__ Hy = p.F[4];
    const S *__restrict__ Hz = p.F[5];
    const float *__restrict__ eps = p.eps;
    unsigned long long pm;
    unsigned sm;
    column_masks(p, i, j, false, pm, sm);
    const bool xyin = i >= 3 && i <= nx - 2 && j >= 3 && j <= ny - 2;
    const Coef<T> Ax = p.A[0], Ay = p.A[1], Az = p.A[2];
    const double t_half = ((double)p.step + 0.5) * p.dt;
    long long o = (long long)k0 * p.sz + (long long)j * p.sy + i;
    // plane-k carries: Hx, Hy at (i,j,k) and eps at the four cells (i..i+1, j..j+1, k)
    T hxc = ldg_s(Hx + o), hyc = ldg_s(Hy + o);
    float f00 = __ldg(eps + o), f10 = __ldg(eps + o + 1), f01 = __ldg(eps + o + p.sy), f11 = __ldg(eps + o + 1 + p.sy);
    for (int k = k0; k < k1; ++k, o += p.sz) {
        const bool fast = xyin && k >= 3 && k <= nz - 2 && !(pm && probe_here(p, pm, k)) && !(sm && source_here(p, sm, k));
        // next plane (k+1) always exists inside the padded array for k <= nz
        const bool has_next = k + 1 < nz + 2;
        const T hxn = has_next ? ldg_s(Hx + o + p.sz) : T(0);
        const T hyn = has_next ? ldg_s(Hy + o + p.sz) : T(0);
        const float e00 = has_next ? __ldg(eps + o + p.sz) : 0.f;
        const float e10 = has_next ? __ldg(eps + o + p.sz + 1) : 0.f;
        const float e01 = has_next ? __ldg(eps + o + p.sz + p.sy) : 0.f;
        const float e11 = has_next ? __ldg(eps + o + p.sz + p.sy + 1) : 0.f;
        if (fast) {
            const T hzc = ldg_s(Hz + o);
            const T hz_jp = ldg_s(Hz + o + p.sy);
            const T hz_ip = ldg_s(Hz + o + 1);
            const T hx_jp = ldg_s(Hx + o + p.sy);
            const T hy_ip = ldg_s(Hy + o + 1);
            typename AccOf<T, S>::type ax, ay, az;
            ax.add(Ay, hz_jp - hzc); ax.add(Az, hyn - hyc, T(-1));
            ay.add(Az, hxn - hxc);   ay.add(Ax, hz_ip - hzc, T(-1));
            az.add(Ax, hy_ip - hyc); az.add(Ay, hx_jp - hxc, T(-1));
            // node sums in the association of cell_sum: Ex (m, +sy, +sz, +sy+sz),
            // Ey (m, +1, +sz, +1+sz), Ez (m, +1, +sy, +1+sy)
            const T sx = (T(f00) + T(f01)) + (T(e00) + T(e01));
            const T sy = (T(f00) + T(f10)) + (T(e00) + T(e10));
            const T sz = (T(f00) + T(f10)) + (T(f01) + T(f11));
            st_s(Ex + o, ld_s(Ex + o) + scaled_increment(ax, sx));
            st_s(Ey + o, ld_s(Ey + o) + scaled_increment(ay, sy));
            st_s(Ez + o, ld_s(Ez + o) + scaled_increment(az, sz));
        } else {
            const int idx[3] = {i, j, k};
            if (i <= nx + 1 && j <= ny && k <= nz) {          // Ex (x-, y+, z+)
                const T en = quant<S>(e_node<T, 0, MUVAR>(p, idx, o, ld_s(Ex + o), sm, t_half));
                st_s(Ex + o, en);
                if (pm) write_probes(p, pm, 0, k, en);
            }
            if (i <= nx && j <= ny + 1 && k <= nz) {          // Ey (x+, y-, z+)
                const T en = quant<S>(e_node<T, 1, MUVAR>(p, idx, o, ld_s(Ey + o), sm, t_half));
                st_s(Ey + o, en);
                if (pm) write_probes(p, pm, 1, k, en);
            }
            if (i <= nx && j <= ny && k <= nz + 1) {          // Ez (x+, y+, z-)
                const T en = quant<S>(e_node<T, 2, MUVAR>(p, idx, o, ld_s(Ez + o), sm, t_half));
                st_s(Ez + o, en);
                if (pm) write_probes(p, pm, 2, k, en);
            }
        }
        hxc = hxn; hyc = hyn;
        f00 = e00; f10 = e10; f01 = e01; f11 = e11;
    }
}

// Fixed-order sum of the per-CTA energy partials (one CTA, deterministic).
__global__ void __launch_bounds__(256) energy_finalize(const double *__restrict__ partials, long long n,
                                                        double *__restrict__ out)
{
    __shared__ double red[256];
    double v = 0.0;
    for (long long q = threadIdx.x; q < n; q += 256) v += partials[q];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = 0.5 * red[0];
}

// FP16 field storage: natural-extent FP32 array (e0 x e1 x e2, x fastest) in,
// padded stored values (value / scale, rounded to nearest) out, and back.
__global__ void put_field_h(const float *__restrict__ src, int e0, int e1, int e2, __half *__restrict__ dst,
                            long long sy, long long sz, float inv_scale)
{
    const long long total = (long long)e0 * e1 * e2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % e0);
        const int j = (int)((q / e0) % e1);
        const int k = (int)(q / ((long long)e0 * e1));
        dst[(long long)k * sz + (long long)j * sy + i] = __float2half_rn(src[q] * inv_scale);
    }
}
__global__ void get_field_h(const __half *__restrict__ src, int e0, int e1, int e2, long long sy, long long sz,
                            float scale, float *__restrict__ dst)
{
    const long long total = (long long)e0 * e1 * e2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % e0);
        const int j = (int)((q / e0) % e1);
        const int k = (int)(q / ((long long)e0 * e1));
        dst[q] = __half2float(src[(long long)k * sz + (long long)j * sy + i]) * scale;
    }
}

// Ghost-padded cell array (coefficient build, once per grid): padded (cx+1,
// cy+1, cz+1) holds cell (cx, cy, cz); ghost layers repeat the nearest cell.
__global__ void pad_cells(const float *__restrict__ cells, int nx, int ny, int nz, float fill,
                          float *__restrict__ out, long long sy, long long sz)
{
    const long long total = (long long)(nx + 2) * (ny + 2) * (nz + 2);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % (nx + 2));
        const int j = (int)((q / (nx + 2)) % (ny + 2));
        const int k = (int)(q / ((long long)(nx + 2) * (ny + 2)));
        float v = fill;
        if (cells) {
            const int cx = min(max(i - 1, 0), nx - 1);
            const int cy = min(max(j - 1, 0), ny - 1);
            const int cz = min(max(k - 1, 0), nz - 1);
            v = cells[((long long)cz * ny + cy) * nx + cx];
        }
        out[(long long)k * sz + (long long)j * sy + i] = v;
    }
}

}  // namespace sbp
