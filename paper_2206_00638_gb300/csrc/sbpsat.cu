// Host side of the C ABI declared in include/sbpsat.h: validation, memory
// layout, coefficient build and kernel launches of the SBP-SAT FDTD leapfrog.
//
// Memory layout in HBM: every field (and the ghost-padded eps_r / mu_r cell
// arrays) uses one common padded shape (nz+2) x (ny+2) x pitch, pitch =
// nx+2 rounded up to 8 elements so each row starts on a 32-byte sector, plus
// one slack plane so that +1 / +row / +plane neighbour reads of the last
// plane stay inside the allocation.  One linear offset o = k*sz + j*sy + i
// addresses node (i, j, k) of every component; positions outside a
// component's natural extents (Table I) stay zero.
//
// Two step paths.  FP32 blocks with uniform mu and at least 8 cells per axis
// keep two field sets and advance with three launches per step (band_h,
// fused_interior, band_e: old set -> new set, then swap).  Everything else
// (FP64, varying mu, energy-monitor steps, the half-step calls) uses the
// in-place h_update / e_update pair on the current set.
#include <cuda_runtime.h>

#include <cfloat>
#include <climits>
#include <cstdint>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sbpsat.h"
#include "kernels.cuh"
#include "fused.cuh"

namespace {

constexpr double kC0 = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.25663706212e-6;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Makes `device` current for the duration of a scope (an entry point) and
// puts the caller's current device back on exit; device < 0 only saves and
// restores (for entry points that visit several devices).
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int device)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (device >= 0 && device != prev) cudaSetDevice(device);
    }
    ~DeviceGuard()
    {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

// NVTX range for the duration of a scope (visible in a profiler's timeline;
// a no-op when no tool is attached).
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
};

}  // namespace

struct sbp_sim {
    int prec = SBP_FP32;
    int n[3] = {0, 0, 0};
    double h[3] = {0, 0, 0};
    double dt = 0;
    int face[6] = {0, 0, 0, 0, 0, 0};
    int energy_every = 0;
    int flags = 0;
    bool fdtd = false;                    // Yee FDTD comparator (SBP_FLAG_FDTD)
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t esize = 4;                     // bytes per stored field element
    size_t psize = 4;                     // bytes per probe sample (the arithmetic type)
    double fscale[2] = {1.0, 1.0};        // physical value = stored value * fscale[E / H] (FP16 storage)
    long long sy = 0, sz = 0;
    size_t field_elems = 0;               // elements per padded array, slack included
    void *set[2][6] = {{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr},
                       {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr}};
    int cur = 0;                          // index of the set holding the current fields
    bool fused_ok = false;                // second set allocated, fused path usable
    bool fused_step = false;              // this step runs the fused path (set during a step)
    int *error_flag = nullptr;            // device flag raised by a pipeline wait that gave up
    sbp::FusedMaps maps[2];               // TMA tensor maps reading set 0 / set 1
    int fused_kchunk = 32;
    int fused_rows = sbp::kFTY;           // tile rows of the one-pass step (tile_valid)
    int fused_width = sbp::kFTX;          // tile columns of the one-pass step (64 or 128)
    dim3 fused_grid;
    bool async_setup = false;             // caller keeps host inputs alive: no stream syncs in setup
    cudaStream_t side = nullptr;          // band_h runs here, concurrently with fused_interior
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    sbp::Band band_hb, band_eb;
    float *eps = nullptr;
    float *mu = nullptr;
    double *partials = nullptr;
    long long npartials = 0;
    double *noalloc_partials = nullptr;   // device address of the library's fixed partial-sum array
    double *escalar = nullptr;
    sbp_sim *nbr[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int nbr_face[6] = {-1, -1, -1, -1, -1, -1};
    sbp_sim *nbr2[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};   // phase pair partner
    double nbr_w[6][2] = {{1, 0}, {1, 0}, {1, 0}, {1, 0}, {1, 0}, {1, 0}};
    std::vector<sbp::Src> src;
    std::vector<sbp::Prb> prb;
    void *probe_buf = nullptr;
    long long probe_cap = 0, probe_base = 0;
    double *eseries = nullptr;
    long long eseries_cap = 0, eseries_count = 0;
    long long step = 0;
    void *workspace = nullptr;
    bool own_ws = false;
    int kchunk = 8;
    dim3 grid;
};

namespace {

struct Layout {
    long long sy, sz;
    size_t field_elems;
    size_t esize;
    size_t field_bytes, cell_bytes, partial_bytes;
    long long npartials;
    int kchunk;
    dim3 grid;
    bool fused;
    int fused_kchunk;
    int fused_rows;
    int fused_width;
    dim3 fused_grid;
    size_t total;
};

// One-pass tiles: 64 columns by 8 or 16 rows (8 or 16 warps), or 128 columns
// by 8 or 12 rows (16 or 24 warps, two per row); the larger ones use most of
// an SM's shared memory.
bool tile_valid(int width, int rows)
{
    return (width == 64 && (rows == 8 || rows == 16)) || (width == 128 && (rows == 8 || rows == 12));
}

// Grid of the one-pass step for tiles of `width` x `rows` H nodes and z-blocks
// of `depth` planes.
dim3 fused_dims(const int n[3], int width, int rows, int depth)
{
    const int tx = (n[0] - 5 + width - 2) / (width - 1);
    const int ty = (n[1] - 5 + rows - 2) / (rows - 1);
    return dim3(tx, ty, (n[2] - 5 + depth - 1) / depth);
}

bool desc_valid(const sbp_grid_desc *d)
{
    if (!d) return false;
    if (d->nx < 4 || d->ny < 4 || d->nz < 4) return false;
    if (!(d->dx > 0) || !(d->dy > 0) || !(d->dz > 0)) return false;
    if (!(d->cfl_fraction > 0)) return false;
    if (d->cfl_fraction > 1.0 && !(d->flags & SBP_FLAG_ALLOW_UNSTABLE)) return false;
    if (d->precision != SBP_FP32 && d->precision != SBP_FP64 && d->precision != SBP_FP32_FP16STORE) return false;
    for (int q = 0; q < 2; q++)
        if (!(d->field_scale[q] >= 0.0) || !std::isfinite(d->field_scale[q])) return false;
    for (int f = 0; f < 6; f++)
        if (d->face[f] < SBP_PEC || d->face[f] > SBP_INTERFACE) return false;
    if (d->energy_every < 0) return false;
    if (d->flags & ~(SBP_FLAG_ALLOW_UNSTABLE | SBP_FLAG_FDTD | SBP_FLAG_TEST_WAIT_TIMEOUT)) return false;
    if (d->flags & SBP_FLAG_FDTD) {
        for (int f = 0; f < 6; f++)
            if (d->face[f] != SBP_PEC) return false;
        if (d->energy_every != 0 || d->precision == SBP_FP64 || d->mu_r || d->nx < 8 || d->ny < 8 || d->nz < 8)
            return false;
    }
    const long long cells = (long long)d->nx * d->ny * d->nz;
    if (cells > (1ll << 34)) return false;
    // every cell finite and >= 1e-3 (NaN fails both comparisons); a branch-free
    // pass, so that the compiler vectorises it (a 512^3 grid has 1.3e8 cells)
    for (const float *m : {d->eps_r, d->mu_r}) {
        if (!m) continue;
        unsigned bad = 0u;
        for (long long q = 0; q < cells; q++) {
            const float v = m[q];
            bad |= (unsigned)!(v >= 1e-3f) | (unsigned)!(v <= FLT_MAX);
        }
        if (bad) return false;
    }
    return true;
}

// tiles chosen by sbp_autotune, per grid shape and precision
struct TileChoice {
    int depth = 0, rows = 0, width = 0;    // depth 0: none recorded
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, TileChoice> g_tuned;
bool g_tune_file_read = false;

// Optional persistence: SBP_TUNE_CACHE names a file of JSON lines
// {"nx": .., "ny": .., "nz": .., "precision": .., "depth": .., "rows": .., "width": ..}
// (a line without "rows" means 8, without "width" 64), read once and appended
// to by every tuning.  Caller holds g_tune_mu.
void read_tune_file()
{
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char *path = std::getenv("SBP_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[256];
    while (std::fgets(line, sizeof(line), f)) {
        int nx, ny, nz, prec, depth, rows = sbp::kFTY, width = sbp::kFTX;
        const int got = std::sscanf(line,
                                    " {\"nx\": %d, \"ny\": %d, \"nz\": %d, \"precision\": %d, \"depth\": %d, "
                                    "\"rows\": %d, \"width\": %d}",
                                    &nx, &ny, &nz, &prec, &depth, &rows, &width);
        if (got >= 5 && depth > 0 && tile_valid(width, rows)) {
            TileChoice t;
            t.depth = depth; t.rows = rows; t.width = width;
            g_tuned[std::make_tuple(nx, ny, nz, prec)] = t;
        }
    }
    std::fclose(f);
}

void append_tune_file(int nx, int ny, int nz, int prec, const TileChoice &t)
{
    const char *path = std::getenv("SBP_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"nx\": %d, \"ny\": %d, \"nz\": %d, \"precision\": %d, \"depth\": %d, \"rows\": %d, "
                 "\"width\": %d}\n",
                 nx, ny, nz, prec, t.depth, t.rows, t.width);
    std::fclose(f);
}

// Tile chosen by sbp_autotune for this shape and precision (depth 0 if none).
TileChoice tuned_tile(const sbp_grid_desc *d)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    read_tune_file();
    auto it = g_tuned.find(std::make_tuple(d->nx, d->ny, d->nz, d->precision));
    return it == g_tuned.end() ? TileChoice() : it->second;
}

Layout make_layout(const sbp_grid_desc *d)
{
    Layout L;
    L.esize = d->precision == SBP_FP64 ? 8 : d->precision == SBP_FP32_FP16STORE ? 2 : 4;
    L.sy = (long long)round_up((size_t)d->nx + 2, 8);
    L.sz = L.sy * (d->ny + 2);
    L.field_elems = (size_t)L.sz * (d->nz + 3);          // nz+2 planes + one slack plane
    L.field_bytes = round_up(L.field_elems * L.esize, 256);
    L.cell_bytes = round_up(L.field_elems * sizeof(float), 256);
    const int gx = (d->nx + 2 + sbp::kBlockX - 1) / sbp::kBlockX;
    const int gy = (d->ny + 2 + sbp::kBlockY - 1) / sbp::kBlockY;
    // enough z-chunks to fill the GPU several times over, at least 8 planes each
    const long long planes = d->nz + 2;
    const long long want_gz = std::max(1ll, (4 * 152 * 4 + (long long)gx * gy - 1) / ((long long)gx * gy));
    int kc = (int)std::max(8ll, (planes + want_gz - 1) / want_gz);
    if (const char *env = std::getenv("SBP_KCHUNK")) {
        const int v = std::atoi(env);
        if (v > 0) kc = v;
    }
    L.kchunk = kc;
    const int gz = (int)((planes + kc - 1) / kc);
    L.grid = dim3(gx, gy, gz);
    L.npartials = (long long)gx * gy * gz;
    L.partial_bytes = round_up((size_t)L.npartials * sizeof(double), 256);
    // (the one-pass kernel addresses a plane with 32-bit offsets)
    L.fused = d->precision != SBP_FP64 && !d->mu_r && d->nx >= 8 && d->ny >= 8 && d->nz >= 8 &&
              L.sz < (1ll << 31) && !std::getenv("SBP_NO_FUSED");
    L.fused_kchunk = 32;
    L.fused_rows = sbp::kFTY;
    L.fused_width = sbp::kFTX;
    L.fused_grid = dim3(1, 1, 1);
    if (L.fused) {
        const int tx = (d->nx - 5 + sbp::kFTX - 2) / (sbp::kFTX - 1);
        const int ty = (d->ny - 5 + sbp::kFTY - 2) / (sbp::kFTY - 1);
        const long long target = 4ll * 2 * 152;        // about four waves of two CTAs per SM
        const long long chunks = std::max(1ll, (target + (long long)tx * ty - 1) / ((long long)tx * ty));
        int kcf = (int)std::max(8ll, ((long long)(d->nz - 5) + chunks - 1) / chunks);
        const TileChoice tt = tuned_tile(d);
        int rows = sbp::kFTY, width = sbp::kFTX;
        if (tt.depth) { kcf = tt.depth; rows = tt.rows; width = tt.width; }
        if (const char *env = std::getenv("SBP_FUSED_KCHUNK")) {
            const int v = std::atoi(env);
            if (v > 0) kcf = v;
        }
        if (const char *env = std::getenv("SBP_FUSED_WIDTH")) {
            const int v = std::atoi(env);
            if (v == 64 || v == 128) width = v;
        }
        if (const char *env = std::getenv("SBP_FUSED_ROWS")) {
            const int v = std::atoi(env);
            if (tile_valid(width, v)) rows = v;
        }
        if (!tile_valid(width, rows)) rows = sbp::kFTY;
        L.fused_kchunk = kcf;
        L.fused_rows = rows;
        L.fused_width = width;
        const int nn[3] = {d->nx, d->ny, d->nz};
        L.fused_grid = fused_dims(nn, width, rows, kcf);
        (void)tx;
        (void)ty;
    }
    L.total = (L.fused ? 12 : 6) * L.field_bytes + L.cell_bytes * (d->mu_r ? 2 : 1) + L.partial_bytes + 256 + 256;
    return L;
}

int cuda_fail(cudaError_t e)
{
    if (e == cudaErrorMemoryAllocation) return SBP_ENOMEM;
    return SBP_ECUDA;
}

// On failure, also consume the runtime's last-error slot so that a
// non-sticky error is not reported again by a later, unrelated call.
#define SBP_CUDA(call)                          \
    do {                                        \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) {                \
            (void)cudaGetLastError();           \
            return cuda_fail(e_);               \
        }                                       \
    } while (0)

// cuTensorMapEncodeTiled, fetched from the driver at run time (no link-time
// dependency on libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

// 3D map over a padded array of 4-byte (FP32) or 2-byte (FP16) elements:
// dims (pitch, ny+2, nz+2), box (bx, rows, 1).
int encode_one(CUtensorMap *m, void *base, const sbp_sim *s, int rows, int esize, int bx)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return SBP_ECUDA;
    const cuuint64_t dims[3] = {(cuuint64_t)s->sy, (cuuint64_t)(s->n[1] + 2), (cuuint64_t)(s->n[2] + 2)};
    const cuuint64_t strides[2] = {(cuuint64_t)s->sy * esize, (cuuint64_t)s->sz * esize};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = fn(m, dt, 3, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SBP_OK : SBP_ECUDA;
}

// TMA maps of both field sets for the current tile: E boxes of rows+1 rows
// (y0-1 .. y0+rows-1), H and eps boxes of rows rows, all width + 16 bytes wide.
int encode_maps(sbp_sim *s)
{
    const int es = (int)s->esize;
    const bool wide = s->fused_width == 128;
    const int bx = es == 2 ? (wide ? sbp::FusedGeom<__half, 8, 128>::kBX : sbp::FusedGeom<__half>::kBX)
                           : (wide ? sbp::FusedGeom<float, 8, 128>::kBX : sbp::FusedGeom<float>::kBX);
    const int rows = s->fused_rows;
    for (int set = 0; set < 2; set++) {
        for (int f = 0; f < 3; f++) {
            int rc = encode_one(&s->maps[set].e[f], s->set[set][f], s, rows + 1, es, bx);
            if (rc) return rc;
            rc = encode_one(&s->maps[set].h[f], s->set[set][3 + f], s, rows, es, bx);
            if (rc) return rc;
        }
        int rc = encode_one(&s->maps[set].eps, s->eps, s, rows, 4, bx);
        if (rc) return rc;
    }
    return SBP_OK;
}

int setup(sbp_sim *s, const sbp_grid_desc *d, const Layout &L, char *ws)
{
    s->prec = d->precision;
    s->n[0] = d->nx; s->n[1] = d->ny; s->n[2] = d->nz;
    s->h[0] = d->dx; s->h[1] = d->dy; s->h[2] = d->dz;
    s->dt = d->cfl_fraction / (kC0 * std::sqrt(1.0 / (d->dx * d->dx) + 1.0 / (d->dy * d->dy) + 1.0 / (d->dz * d->dz)));
    for (int f = 0; f < 6; f++) s->face[f] = d->face[f];
    s->energy_every = d->energy_every;
    s->flags = d->flags;
    s->fdtd = (d->flags & SBP_FLAG_FDTD) != 0;
    if (s->fdtd && !L.fused) return SBP_EINVAL;   // the comparator runs in the one-pass + band kernels only
    s->esize = L.esize;
    s->psize = d->precision == SBP_FP64 ? 8 : 4;
    if (d->precision == SBP_FP32_FP16STORE) {
        // default scales: E in V/m as is, H as eta0 * H (the two then have
        // comparable magnitudes in a wave)
        s->fscale[0] = d->field_scale[0] > 0 ? d->field_scale[0] : 1.0;
        s->fscale[1] = d->field_scale[1] > 0 ? d->field_scale[1] : 1.0 / std::sqrt(kMu0 / kEps0);
    }
    s->sy = L.sy; s->sz = L.sz;
    s->field_elems = L.field_elems;
    s->kchunk = L.kchunk;
    s->grid = L.grid;
    s->npartials = L.npartials;
    s->fused_ok = L.fused;
    s->fused_kchunk = L.fused_kchunk;
    s->fused_rows = L.fused_rows;
    s->fused_width = L.fused_width;
    s->fused_grid = L.fused_grid;
    char *p = ws;
    for (int set = 0; set < (L.fused ? 2 : 1); set++)
        for (int c = 0; c < 6; c++) { s->set[set][c] = p; p += L.field_bytes; }
    s->eps = reinterpret_cast<float *>(p); p += L.cell_bytes;
    if (d->mu_r) { s->mu = reinterpret_cast<float *>(p); p += L.cell_bytes; }
    s->partials = reinterpret_cast<double *>(p); p += L.partial_bytes;
    s->escalar = reinterpret_cast<double *>(p); p += 256;
    s->error_flag = reinterpret_cast<int *>(p);
    SBP_CUDA(cudaMemsetAsync(s->error_flag, 0, sizeof(int), s->stream));

    // coefficient build (a1): ghost-padded cell arrays on the device.  The
    // caller's cells are staged through the (still unused) Hx array.
    const size_t ncell = (size_t)d->nx * d->ny * d->nz;
    const int threads = 256;
    const int blocks = (int)std::min<long long>(4096, (L.field_elems + threads - 1) / threads);
    for (int m = 0; m < 2; m++) {
        const float *host = m == 0 ? d->eps_r : d->mu_r;
        float *dst = m == 0 ? s->eps : s->mu;
        if (m == 1 && !d->mu_r) break;
        float *stage = nullptr;
        if (host) {
            stage = static_cast<float *>(s->set[0][3]);
            SBP_CUDA(cudaMemcpyAsync(stage, host, ncell * sizeof(float), cudaMemcpyHostToDevice, s->stream));
        }
        SBP_CUDA(cudaMemsetAsync(dst, 0, L.field_elems * sizeof(float), s->stream));
        sbp::pad_cells<<<blocks, threads, 0, s->stream>>>(stage, d->nx, d->ny, d->nz, 1.0f, dst, L.sy, L.sz);
        SBP_CUDA(cudaGetLastError());
        if (!s->async_setup) SBP_CUDA(cudaStreamSynchronize(s->stream));   // host cells may be released after return
    }
    for (int set = 0; set < (L.fused ? 2 : 1); set++)
        for (int c = 0; c < 6; c++) SBP_CUDA(cudaMemsetAsync(s->set[set][c], 0, L.field_elems * L.esize, s->stream));
    if (!s->async_setup) SBP_CUDA(cudaStreamSynchronize(s->stream));
    if (L.fused) {
        int rc = encode_maps(s);
        if (rc) return rc;
        SBP_CUDA(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
        SBP_CUDA(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
        SBP_CUDA(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
        // The one-pass step covers H on [3, n-2] and E on [3, n-3] per axis.
        // The H band also takes the first interior layer (H on [4, n-3] is
        // left to the one-pass step alone): an E band node reads H at most
        // one node inward along each axis (D+ rows 0..2 read H 0..3, row n-2
        // reads H n-2, n-1), so band E depends on band H only and both run
        // beside the one-pass step.  Both kernels write that layer with the
        // same formula and the same rounding, hence the same bits.
        for (int phase = 0; phase < 2; phase++) {
            sbp::Band &b = phase == 0 ? s->band_hb : s->band_eb;
            b.lo = phase == 0 ? 4 : 3;
            for (int a = 0; a < 3; a++) b.hi[a] = s->n[a] - 3;
            // warps: 32-node x-row segments (x in [lo, hi_x]) for the z and
            // y slabs, 4 x-end nodes x 8 rows for the x slab (both x-ends at
            // most 4 wide; segments start at x = 0, so lo < 32)
            if (b.lo > 4 || s->n[0] + 1 - b.hi[0] > 4) return SBP_EINVAL;
            const long long segs = b.hi[0] / 32 + 1, ey = s->n[1] + 2, ez = s->n[2] + 2;
            const long long zplanes = b.lo + (s->n[2] + 1 - b.hi[2]);
            const long long yrows = b.lo + (s->n[1] + 1 - b.hi[1]);
            const long long jin = b.hi[1] - b.lo + 1, xgroups = (ey + 7) / 8;
            const long long wz = zplanes * jin * segs, wy = ez * yrows * segs, wx = ez * xgroups * 2;
            if (wz + wy + wx >= (1ll << 32) - 8) return SBP_EINVAL;
            b.segs = (unsigned)segs;
            b.zplanes = (unsigned)zplanes;
            b.yrows = (unsigned)yrows;
            b.jin = (unsigned)jin;
            b.xgroups = (unsigned)xgroups;
            b.wz = (unsigned)wz;
            b.wy = (unsigned)wy;
            b.wx = (unsigned)wx;
            b.ctas = (unsigned)((wz + wy + wx + 7) / 8);
        }
    }
    return SBP_OK;
}

template <typename T>
sbp::Coef<T> split(double v)
{
    sbp::Coef<T> c;
    c.hi = (T)v;
    c.lo = (T)(v - (double)c.hi);
    return c;
}

// Kernel parameters reading E from field set eset and H from set hset.
// Interface partners: E from the partner's current set; H from the set the
// partner's H^{n+1/2} lands in this step (its new set when it runs fused).
template <typename T, typename S = T>
int make_params(const sbp_sim *s, sbp::Params<T, S> &p, int eset, int hset)
{
    std::memset(&p, 0, sizeof(p));
    for (int c = 0; c < 3; c++) p.F[c] = static_cast<S *>(s->set[eset][c]);
    for (int c = 3; c < 6; c++) p.F[c] = static_cast<S *>(s->set[hset][c]);
    p.eps = s->eps;
    p.mu = s->mu;
    for (int a = 0; a < 3; a++) p.n[a] = s->n[a];
    p.sy = s->sy;
    p.sz = s->sz;
    for (int f = 0; f < 6; f++) {
        p.face[f] = s->face[f];
        if (s->face[f] == SBP_INTERFACE) {
            const sbp_sim *nb = s->nbr[f];
            if (!nb) return SBP_ESTATE;
            const int nh = nb->fused_step ? nb->cur ^ 1 : nb->cur;
            for (int c = 0; c < 3; c++) p.link[f].F[c] = nb->set[nb->cur][c];
            for (int c = 3; c < 6; c++) p.link[f].F[c] = nb->set[nh][c];
            if (const sbp_sim *n2 = s->nbr2[f]) {
                const int nh2 = n2->fused_step ? n2->cur ^ 1 : n2->cur;
                for (int c = 0; c < 3; c++) p.link[f].G[c] = n2->set[n2->cur][c];
                for (int c = 3; c < 6; c++) p.link[f].G[c] = n2->set[nh2][c];
                p.link[f].w[0] = s->nbr_w[f][0];
                p.link[f].w[1] = s->nbr_w[f][1];
            }
            p.link[f].sy = nb->sy;
            p.link[f].sz = nb->sz;
            p.link[f].n_norm = nb->n[f / 2];
            p.link[f].side = (s->nbr_face[f] % 2) ? 1 : -1;
        }
    }
    // stored fields are E / sE and H / sH: the H update takes B sE / sH, the
    // E update A sH / sE and the source term AJ / sE (all 1 unless FP16 storage)
    const double bscale = s->mu ? 2.0 : 1.0;
    const double sE = s->fscale[0], sH = s->fscale[1];
    for (int a = 0; a < 3; a++) {
        p.B[a] = split<T>(bscale * s->dt / (kMu0 * s->h[a]) * (sE / sH));
        p.A[a] = split<T>(4.0 * s->dt / (kEps0 * s->h[a]) * (sH / sE));
        p.h[a] = s->h[a];
    }
    p.AJ = split<T>(4.0 * s->dt / kEps0 / sE);
    p.fscale[0] = (T)sE;
    p.fscale[1] = (T)sH;
    p.uB = (T)(sH / sE);
    p.uA = (T)(sE / sH);
    p.dt = s->dt;
    p.eta0 = std::sqrt(kMu0 / kEps0);
    p.eps0 = kEps0;
    p.mu0 = kMu0;
    p.nsrc = (int)s->src.size();
    for (int q = 0; q < p.nsrc; q++) p.src[q] = s->src[q];
    p.nprb = (int)s->prb.size();
    for (int q = 0; q < p.nprb; q++) p.prb[q] = s->prb[q];
    p.probe_buf = static_cast<T *>(s->probe_buf);   // samples in the arithmetic type
    p.probe_cap = s->probe_buf ? s->probe_cap : 0;
    p.probe_slot = s->step - s->probe_base;
    p.step = s->step;
    p.partials = s->partials;
    p.kchunk = s->kchunk;
    p.fdtd = s->fdtd ? 1 : 0;
    return SBP_OK;
}

template <typename T, typename S>
int launch_h(const sbp_sim *s, bool energy, bool store)
{
    sbp::Params<T, S> p;
    int rc = make_params<T, S>(s, p, s->cur, s->cur);
    if (rc) return rc;
    const dim3 block(sbp::kBlockX, sbp::kBlockY);
    const bool muv = s->mu != nullptr;
    if (!energy) {
        if (muv) sbp::h_update<T, S, false, true, true><<<s->grid, block, 0, s->stream>>>(p);
        else sbp::h_update<T, S, false, true, false><<<s->grid, block, 0, s->stream>>>(p);
    } else if (store) {
        if (muv) sbp::h_update<T, S, true, true, true><<<s->grid, block, 0, s->stream>>>(p);
        else sbp::h_update<T, S, true, true, false><<<s->grid, block, 0, s->stream>>>(p);
    } else {
        if (muv) sbp::h_update<T, S, true, false, true><<<s->grid, block, 0, s->stream>>>(p);
        else sbp::h_update<T, S, true, false, false><<<s->grid, block, 0, s->stream>>>(p);
    }
    SBP_CUDA(cudaGetLastError());
    return SBP_OK;
}

template <typename T, typename S>
int launch_e(const sbp_sim *s)
{
    sbp::Params<T, S> p;
    int rc = make_params<T, S>(s, p, s->cur, s->cur);
    if (rc) return rc;
    const dim3 block(sbp::kBlockX, sbp::kBlockY);
    if (s->mu) sbp::e_update<T, S, true><<<s->grid, block, 0, s->stream>>>(p);
    else sbp::e_update<T, S, false><<<s->grid, block, 0, s->stream>>>(p);
    SBP_CUDA(cudaGetLastError());
    return SBP_OK;
}

int launch_h_any(const sbp_sim *s, bool energy, bool store)
{
    if (s->prec == SBP_FP64) return launch_h<double, double>(s, energy, store);
    if (s->prec == SBP_FP32_FP16STORE) return launch_h<float, __half>(s, energy, store);
    return launch_h<float, float>(s, energy, store);
}
int launch_e_any(const sbp_sim *s)
{
    if (s->prec == SBP_FP64) return launch_e<double, double>(s);
    if (s->prec == SBP_FP32_FP16STORE) return launch_e<float, __half>(s);
    return launch_e<float, float>(s);
}

// Parameters of the one-pass interior step reading set `old`, writing set old^1.
template <typename S>
int make_fused_params(const sbp_sim *s, int old, sbp::FusedParamsT<S> &fp)
{
    sbp::Params<float, S> p;
    int rc = make_params<float, S>(s, p, old, old);
    if (rc) return rc;
    S **ns = reinterpret_cast<S **>(const_cast<void **>(s->set[old ^ 1]));
    std::memset(&fp, 0, sizeof(fp));
    for (int c = 0; c < 6; c++) fp.out[c] = ns[c];
    fp.pscale[0] = p.fscale[0];
    fp.pscale[1] = p.fscale[1];
    for (int a = 0; a < 3; a++) { fp.n[a] = s->n[a]; fp.B[a] = p.B[a]; fp.A[a] = p.A[a]; }
    fp.sy = s->sy;
    fp.sz = s->sz;
    fp.AJ = p.AJ;
    fp.dt = p.dt;
    fp.nsrc = p.nsrc;
    for (int q = 0; q < p.nsrc; q++) fp.src[q] = p.src[q];
    fp.nprb = p.nprb;
    for (int q = 0; q < p.nprb; q++) fp.prb[q] = p.prb[q];
    fp.probe_buf = p.probe_buf;
    fp.probe_cap = p.probe_cap;
    fp.probe_slot = p.probe_slot;
    fp.step = p.step;
    fp.kchunk = s->fused_kchunk;
    fp.error_flag = s->error_flag;
    fp.test_stall = (s->flags & SBP_FLAG_TEST_WAIT_TIMEOUT) ? 1 : 0;
    fp.wait_limit = fp.test_stall ? (1u << 10) : sbp::kWaitLimit;
    return SBP_OK;
}

int set_fused_smem_attr()
{
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !done[dev]) {
        const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
#define SBP_FUSED_ATTR(S, R, W)                                                                               \
        SBP_CUDA(cudaFuncSetAttribute(sbp::fused_interior<true, S, R, W>, attr, sbp::FusedGeom<S, R, W>::kSmem)); \
        SBP_CUDA(cudaFuncSetAttribute(sbp::fused_interior<false, S, R, W>, attr, sbp::FusedGeom<S, R, W>::kSmem))
        SBP_FUSED_ATTR(float, 8, 64);
        SBP_FUSED_ATTR(float, 16, 64);
        SBP_FUSED_ATTR(float, 8, 128);
        SBP_FUSED_ATTR(float, 12, 128);
        SBP_FUSED_ATTR(__half, 8, 64);
        SBP_FUSED_ATTR(__half, 16, 64);
        SBP_FUSED_ATTR(__half, 8, 128);
        SBP_FUSED_ATTR(__half, 12, 128);
#undef SBP_FUSED_ATTR
        SBP_CUDA(cudaFuncSetAttribute(sbp::fused_batched<8>, attr, sbp::FusedGeom<float, 8>::kSmem));
        SBP_CUDA(cudaFuncSetAttribute(sbp::fused_batched<16>, attr, sbp::FusedGeom<float, 16>::kSmem));
        SBP_CUDA(cudaFuncSetAttribute(sbp::persistent_batched, attr, sbp::kFusedSmem));
        done[dev] = true;
    }
    return SBP_OK;
}

template <typename S, int R, int W>
void launch_fused_tile(sbp_sim *s, const sbp::FusedParamsT<S> &fp, int old)
{
    using Gm = sbp::FusedGeom<S, R, W>;
    if (fp.nsrc > 0)
        sbp::fused_interior<true, S, R, W><<<s->fused_grid, Gm::kWarps * 32, Gm::kSmem, s->stream>>>(s->maps[old], fp);
    else
        sbp::fused_interior<false, S, R, W><<<s->fused_grid, Gm::kWarps * 32, Gm::kSmem, s->stream>>>(s->maps[old], fp);
}

// The one-pass interior step (old set -> new set).
template <typename S>
int launch_fused_interior_t(sbp_sim *s)
{
    const int old = s->cur;
    sbp::FusedParamsT<S> fp;
    int rc = make_fused_params<S>(s, old, fp);
    if (rc) return rc;
    rc = set_fused_smem_attr();
    if (rc) return rc;
    if (s->fused_width == 128) {
        if (s->fused_rows == 12) launch_fused_tile<S, 12, 128>(s, fp, old);
        else launch_fused_tile<S, 8, 128>(s, fp, old);
    } else {
        if (s->fused_rows == 16) launch_fused_tile<S, 16, 64>(s, fp, old);
        else launch_fused_tile<S, 8, 64>(s, fp, old);
    }
    SBP_CUDA(cudaGetLastError());
    return SBP_OK;
}

// Band H (old -> new) on stream st.
template <typename S>
int launch_band_h_t(sbp_sim *s, cudaStream_t st)
{
    const int old = s->cur, nw = s->cur ^ 1;
    sbp::Params<float, S> p;
    int rc = make_params<float, S>(s, p, old, old);
    if (rc) return rc;
    const sbp::Band &bh = s->band_hb;
    S **ns = reinterpret_cast<S **>(s->set[nw]);
    sbp::band_h<float, false><<<bh.ctas, 256, 0, st>>>(p, bh, ns[3], ns[4], ns[5]);
    SBP_CUDA(cudaGetLastError());
    return SBP_OK;
}

// Band E from E^n (old) and H^{n+1/2} (new) into the new set, on stream st.
template <typename S>
int launch_band_e_t(sbp_sim *s, cudaStream_t st)
{
    const int old = s->cur, nw = s->cur ^ 1;
    sbp::Params<float, S> p;
    int rc = make_params<float, S>(s, p, old, nw);
    if (rc) return rc;
    const sbp::Band &be = s->band_eb;
    S **ns = reinterpret_cast<S **>(s->set[nw]);
    sbp::band_e<float, false><<<be.ctas, 256, 0, st>>>(p, be, ns[0], ns[1], ns[2]);
    SBP_CUDA(cudaGetLastError());
    return SBP_OK;
}

// The fused path runs for FP32 arithmetic with FP32 or FP16 storage.
int launch_fused_interior_only(sbp_sim *s)
{
    return s->prec == SBP_FP32_FP16STORE ? launch_fused_interior_t<__half>(s) : launch_fused_interior_t<float>(s);
}
int launch_band_h(sbp_sim *s, cudaStream_t st)
{
    return s->prec == SBP_FP32_FP16STORE ? launch_band_h_t<__half>(s, st) : launch_band_h_t<float>(s, st);
}
int launch_band_e(sbp_sim *s, cudaStream_t st)
{
    return s->prec == SBP_FP32_FP16STORE ? launch_band_e_t<__half>(s, st) : launch_band_e_t<float>(s, st);
}

// Fused path, phase 1: the one-pass interior step on the main stream and,
// beside it on the side stream, band H (old -> new) followed by band E when
// `chain_e` (band E of a block whose interface partner is another block waits
// for that partner's band H instead: phase 2).  Joined before returning.
int launch_fused_phase1(sbp_sim *s, bool chain_e)
{
    SBP_CUDA(cudaEventRecord(s->ev_fork, s->stream));
    int rc = launch_fused_interior_only(s);
    if (rc) return rc;
    SBP_CUDA(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
    if ((rc = launch_band_h(s, s->side))) return rc;
    if (chain_e && (rc = launch_band_e(s, s->side))) return rc;
    SBP_CUDA(cudaEventRecord(s->ev_join, s->side));
    SBP_CUDA(cudaStreamWaitEvent(s->stream, s->ev_join, 0));
    return SBP_OK;
}

// Fused path, phase 2 (blocks joined to another block): band E on the main stream.
int launch_fused_phase2(sbp_sim *s) { return launch_band_e(s, s->stream); }

// True when an interface face of s joins it to a block other than itself.
bool linked_to_other(const sbp_sim *s)
{
    for (int f = 0; f < 6; f++)
        if (s->face[f] == SBP_INTERFACE && ((s->nbr[f] && s->nbr[f] != s) || s->nbr2[f])) return true;
    return false;
}

int finalize_energy(const sbp_sim *s, double *dst)
{
    sbp::energy_finalize<<<1, 256, 0, s->stream>>>(s->partials, s->npartials, dst);
    SBP_CUDA(cudaGetLastError());
    return SBP_OK;
}

// Partial sums of sbp_energy_noalloc: a fixed array in this library, so that
// call allocates nothing.  In host code the name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress, looked up when a
// simulation is created, with its device current, and kept in the simulation
// (a device reset invalidates both together).
static __device__ __align__(256) double g_noalloc_partials[SBP_NOALLOC_MAX_PARTIALS];

int noalloc_scratch(double **out)
{
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
    if (e != cudaSuccess || !ptr) {
        (void)cudaGetLastError();
        return SBP_ECUDA;
    }
    *out = static_cast<double *>(ptr);
    return SBP_OK;
}

// The energy query of sbp_energy with the partial sums in `partials` and the
// result written to the device pointer `dst`.
template <typename T, typename S>
int energy_into_t(const sbp_sim *s, double *partials, double *dst)
{
    sbp::Params<T, S> p;
    int rc = make_params<T, S>(s, p, s->cur, s->cur);
    if (rc) return rc;
    p.partials = partials;
    const dim3 block(sbp::kBlockX, sbp::kBlockY);
    if (s->mu) sbp::h_update<T, S, true, false, true><<<s->grid, block, 0, s->stream>>>(p);
    else sbp::h_update<T, S, true, false, false><<<s->grid, block, 0, s->stream>>>(p);
    SBP_CUDA(cudaGetLastError());
    sbp::energy_finalize<<<1, 256, 0, s->stream>>>(partials, s->npartials, dst);
    SBP_CUDA(cudaGetLastError());
    return SBP_OK;
}

int energy_into(const sbp_sim *s, double *partials, double *dst)
{
    if (s->prec == SBP_FP64) return energy_into_t<double, double>(s, partials, dst);
    if (s->prec == SBP_FP32_FP16STORE) return energy_into_t<float, __half>(s, partials, dst);
    return energy_into_t<float, float>(s, partials, dst);
}

int ensure_series(sbp_sim *s, long long need)
{
    if (need <= s->eseries_cap) return SBP_OK;
    long long cap = std::max(need, 2 * s->eseries_cap + 16);
    double *nb = nullptr;
    SBP_CUDA(cudaMalloc(&nb, cap * sizeof(double)));
    SBP_CUDA(cudaMemsetAsync(nb, 0, cap * sizeof(double), s->stream));   // samples not taken read 0
    if (s->eseries && s->eseries_count > 0)
        SBP_CUDA(cudaMemcpyAsync(nb, s->eseries, s->eseries_count * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    SBP_CUDA(cudaStreamSynchronize(s->stream));
    if (s->eseries) cudaFree(s->eseries);
    s->eseries = nb;
    s->eseries_cap = cap;
    return SBP_OK;
}

int extents_of(const sbp_sim *s, int comp, int e[3])
{
    if (comp < 0 || comp > 5) return SBP_EINVAL;
    for (int a = 0; a < 3; a++) e[a] = s->n[a] + (sbp::on_plus(comp, a) ? 1 : 2);
    return SBP_OK;
}

int create_common(const sbp_grid_desc *d, void *stream, void *ws, size_t bytes, bool own, sbp_sim **out,
                  bool async_setup = false, bool validated = false)
{
    if (!out || (!validated && !desc_valid(d))) return SBP_EINVAL;
    *out = nullptr;
    Layout L = make_layout(d);
    sbp_sim *s = new (std::nothrow) sbp_sim();
    if (!s) return SBP_ENOMEM;
    s->async_setup = async_setup;
    cudaGetDevice(&s->device);
    s->stream = static_cast<cudaStream_t>(stream);
    if (own) {
        cudaError_t e = cudaMalloc(&ws, L.total);
        if (e != cudaSuccess) { delete s; return cuda_fail(e); }
        s->own_ws = true;
    } else {
        if (!ws || bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255)) { delete s; return ws ? SBP_ECAPACITY : SBP_EINVAL; }
    }
    s->workspace = ws;
    int rc = noalloc_scratch(&s->noalloc_partials);
    if (!rc) rc = setup(s, d, L, static_cast<char *>(ws));
    if (rc) { if (s->own_ws) cudaFree(ws); delete s; return rc; }
    *out = s;
    return SBP_OK;
}

int check_group(sbp_sim **sims, int nsims)
{
    if (!sims || nsims <= 0) return SBP_EINVAL;
    for (int q = 0; q < nsims; q++) {
        if (!sims[q]) return SBP_EINVAL;
        if (sims[q]->stream != sims[0]->stream) return SBP_EINVAL;
        for (int f = 0; f < 6; f++)
            if (sims[q]->face[f] == SBP_INTERFACE && !sims[q]->nbr[f]) return SBP_ESTATE;
    }
    return SBP_OK;
}

int half_h(sbp_sim **sims, int nsims)
{
    for (int q = 0; q < nsims; q++) {
        sbp_sim *s = sims[q];
        const bool mon = s->energy_every > 0 && (s->step % s->energy_every) == 0;
        if (mon) {
            int rc = ensure_series(s, s->step / s->energy_every + 1);
            if (rc) return rc;
        }
        int rc = launch_h_any(s, mon, true);
        if (rc) return rc;
        if (mon) {
            rc = finalize_energy(s, s->eseries + s->step / s->energy_every);
            if (rc) return rc;
            s->eseries_count = s->step / s->energy_every + 1;
        }
    }
    return SBP_OK;
}

int half_e(sbp_sim **sims, int nsims)
{
    for (int q = 0; q < nsims; q++) {
        int rc = launch_e_any(sims[q]);
        if (rc) return rc;
    }
    for (int q = 0; q < nsims; q++) sims[q]->step++;
    return SBP_OK;
}

int step_group(sbp_sim **sims, int nsims, int64_t nsteps)
{
    Trace trace("sbp_step");
    if (nsteps < 0) return SBP_EINVAL;
    int rc = check_group(sims, nsims);
    if (rc) return rc;
    DeviceGuard dg(sims[0]->device);
    for (int q = 0; q < nsims; q++) {
        sbp_sim *s = sims[q];
        if (s->energy_every > 0) {
            rc = ensure_series(s, (s->step + nsteps) / s->energy_every + 1);
            if (rc) return rc;
        }
    }
    for (int64_t t = 0; t < nsteps; t++) {
        // decide each block's path first: interface partners read it
        for (int q = 0; q < nsims; q++) {
            sbp_sim *s = sims[q];
            const bool mon = s->energy_every > 0 && (s->step % s->energy_every) == 0;
            s->fused_step = s->fused_ok && !mon;
        }
        for (int q = 0; q < nsims; q++) {
            sbp_sim *s = sims[q];
            rc = s->fused_step ? launch_fused_phase1(s, !linked_to_other(s)) : half_h(&s, 1);
            if (rc) return rc;
        }
        for (int q = 0; q < nsims; q++) {
            sbp_sim *s = sims[q];
            if (s->fused_step) {
                if (!linked_to_other(s)) continue;
                rc = launch_fused_phase2(s);
                if (rc) return rc;
            } else {
                rc = launch_e_any(s);
                if (rc) return rc;
            }
        }
        for (int q = 0; q < nsims; q++) {
            sbp_sim *s = sims[q];
            if (s->fused_step) s->cur ^= 1;
            s->fused_step = false;
            s->step++;
        }
    }
    return SBP_OK;
}

// sbp_step with CUDA events around every launch (kernel kinds: 0 h_update,
// 1 e_update, 2 band_h, 3 fused_interior, 4 band_e).
int step_timed(sbp_sim *s, int64_t nsteps, double *avg_ms, int64_t *launches, int n_out)
{
    constexpr int kKinds = 5;
    double tot[kKinds] = {0, 0, 0, 0, 0};
    long long cnt[kKinds] = {0, 0, 0, 0, 0};
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    auto mark = [&](int k) -> int {
        cudaEvent_t e;
        SBP_CUDA(cudaEventCreate(&e));
        SBP_CUDA(cudaEventRecord(e, s->stream));
        ev.push_back(e);
        kind.push_back(k);
        return SBP_OK;
    };
    int rc = SBP_OK;
    for (int64_t t = 0; t < nsteps && !rc; t++) {
        const bool mon = s->energy_every > 0 && (s->step % s->energy_every) == 0;
        s->fused_step = s->fused_ok && !mon && s->face[0] != SBP_INTERFACE && s->face[1] != SBP_INTERFACE &&
                        s->face[2] != SBP_INTERFACE && s->face[3] != SBP_INTERFACE && s->face[4] != SBP_INTERFACE &&
                        s->face[5] != SBP_INTERFACE;
        if (s->fused_step) {
            // the three kernels of a fused step, one after another on the
            // stream so that each is timed alone
            if ((rc = mark(2))) break;
            if ((rc = launch_band_h(s, s->stream))) break;
            if ((rc = mark(-1))) break;
            if ((rc = mark(3))) break;
            if ((rc = launch_fused_interior_only(s))) break;
            if ((rc = mark(-1))) break;
            if ((rc = mark(4))) break;
            if ((rc = launch_fused_phase2(s))) break;
            if ((rc = mark(-1))) break;
            s->cur ^= 1;
        } else {
            if ((rc = mark(0))) break;
            if ((rc = half_h(&s, 1))) break;
            if ((rc = mark(-1))) break;
            if ((rc = mark(1))) break;
            if ((rc = launch_e_any(s))) break;
            if ((rc = mark(-1))) break;
        }
        s->fused_step = false;
        s->step++;
    }
    cudaStreamSynchronize(s->stream);
    for (size_t q = 0; q + 1 < ev.size(); q += 2) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
        tot[kind[q]] += ms;
        cnt[kind[q]]++;
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (int k = 0; k < n_out && k < kKinds; k++) {
        if (avg_ms) avg_ms[k] = cnt[k] ? tot[k] / cnt[k] : 0.0;
        if (launches) launches[k] = cnt[k];
    }
    return rc;
}

int check_error_flag(sbp_sim *s)
{
    if (!s->error_flag) return SBP_OK;
    int v = 0;
    SBP_CUDA(cudaMemcpy(&v, s->error_flag, sizeof(int), cudaMemcpyDeviceToHost));
    return v ? SBP_ETIMEOUT : SBP_OK;
}

// Tile of the one-pass step: width x rows (tile_valid) and z-block depth; a
// new width or row count re-encodes the TMA maps (their boxes have its shape).
int set_tile(sbp_sim *s, int width, int rows, int depth)
{
    if (!tile_valid(width, rows) || depth <= 0) return SBP_EINVAL;
    s->fused_kchunk = depth;
    if (rows != s->fused_rows || width != s->fused_width) {
        s->fused_rows = rows;
        s->fused_width = width;
        int rc = encode_maps(s);
        if (rc) return rc;
    }
    s->fused_grid = fused_dims(s->n, width, rows, depth);
    return SBP_OK;
}

// Average device time of `trials` fused steps that are not committed: each
// writes the whole new field set and this step's probe slot, both of which
// the next real step overwrites, and the current set is left as it was.
int time_trials(sbp_sim *s, int trials, cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    const bool chain = !linked_to_other(s);
    int rc = launch_fused_phase1(s, chain);           // warm-up of this depth
    if (!rc && !chain) rc = launch_fused_phase2(s);
    if (rc) return rc;
    SBP_CUDA(cudaEventRecord(e0, s->stream));
    for (int t = 0; t < trials; t++) {
        if ((rc = launch_fused_phase1(s, chain))) return rc;
        if (!chain && (rc = launch_fused_phase2(s))) return rc;
    }
    SBP_CUDA(cudaEventRecord(e1, s->stream));
    SBP_CUDA(cudaEventSynchronize(e1));
    SBP_CUDA(cudaEventElapsedTime(ms, e0, e1));
    *ms /= (float)trials;
    return SBP_OK;
}

int autotune(sbp_sim *s, int trials, int *chosen, double *best_ms)
{
    Trace trace("sbp_autotune");
    // a block joined to others tunes too: its trial steps read the partners' current
    // fields at the interface and write only this block's spare set
    if (!s->fused_ok) return SBP_ESTATE;
    const int span = s->n[2] - 5;                      // interior E planes of the one-pass step
    std::vector<TileChoice> cand;
    const int shapes[4][2] = {{64, 8}, {64, 16}, {128, 8}, {128, 12}};   // (width, rows)
    for (const auto &sh : shapes) {
        if (sh[1] > 8 && s->n[1] - 5 < sh[1] - 1) continue;      // no full tile of that height
        if (sh[0] > 64 && s->n[0] - 5 < sh[0] - 1) continue;     // nor of that width
        for (int c : {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256})
            if (c <= span || c == 8) {
                TileChoice t;
                t.width = sh[0]; t.rows = sh[1]; t.depth = c;
                cand.push_back(t);
            }
    }
    TileChoice keep;
    keep.width = s->fused_width; keep.rows = s->fused_rows; keep.depth = s->fused_kchunk;
    auto same = [](const TileChoice &a, const TileChoice &b) {
        return a.width == b.width && a.rows == b.rows && a.depth == b.depth;
    };
    if (std::none_of(cand.begin(), cand.end(), [&](const TileChoice &c) { return same(c, keep); }))
        cand.push_back(keep);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SBP_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaEventDestroy(e0);
        return SBP_ECUDA;
    }
    TileChoice best = keep;
    int rc = SBP_OK;
    float best_t = 0.f;
    for (const auto &c : cand) {
        if ((rc = set_tile(s, c.width, c.rows, c.depth))) break;
        float t = 0.f;
        if ((rc = time_trials(s, trials, e0, e1, &t))) break;
        if (best_t == 0.f || t < best_t) { best_t = t; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const TileChoice fin = rc ? keep : best;
    const int rc2 = set_tile(s, fin.width, fin.rows, fin.depth);
    if (rc) return rc;
    if (rc2) return rc2;
    if ((rc = check_error_flag(s))) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        read_tune_file();
        g_tuned[std::make_tuple(s->n[0], s->n[1], s->n[2], s->prec)] = best;
        append_tune_file(s->n[0], s->n[1], s->n[2], s->prec, best);
    }
    if (chosen) *chosen = best.depth;
    if (best_ms) *best_ms = best_t;
    return SBP_OK;
}

}  // namespace

// A batch: many single-block FP32 simulations advanced together, one launch
// per kernel kind per step for all of them (see BatchGrid in fused.cuh).
struct sbp_batch {
    struct Member {
        sbp_sim *s;
        long long target;        // absolute step index at which the member stops
        double *mirror;          // pinned host copy of the latest energy sample (serving), or null
    };
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on (capture runs nothing)
    cudaStream_t side = nullptr;        // band H -> band E beside the one-pass step
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0;
    std::vector<Member> m;
    sbp::BatchGrid *d_grids = nullptr;
    int *d_pre = nullptr;               // four prefix tables of cap+1 ints: fused, band H, band E CTAs,
                                        // persistent-kernel items
    long long *d_counters = nullptr;
    int cap = 0;
    int nf = 0, nh = 0, ne = 0;         // CTAs per launch
    int rows = sbp::kFTY;               // tile rows of the per-step one-pass launch (8 or 16)
    int ni = 0;                         // persistent-kernel items per step
    sbp::BatchGrid *h_grids = nullptr;  // pinned staging of the uploads
    int *h_pre = nullptr;
    long long *h_counters = nullptr;
    cudaEvent_t staged = nullptr;       // the last upload has left the staging buffers
    bool dirty = true;
    bool use_graph = true;
    bool persistent = false;            // one persistent launch per chunk (else three launches per step)
    unsigned *d_sched = nullptr;        // persistent kernel: ticket counter, 2 counters per member, error flag
    int *h_err = nullptr;               // pinned copy of the persistent kernel's error flag
    int resident = 0;                   // CTAs of the persistent kernel resident at once
    cudaGraphExec_t gexec = nullptr;
    long long gK = 0;
    bool gstale = false;                // membership changed since gexec was recorded
};

namespace {

int batch_reserve(sbp_batch *b, int n)
{
    if (n <= b->cap) return SBP_OK;
    const int cap = std::max(n, 2 * b->cap + 4);
    SBP_CUDA(cudaStreamSynchronize(b->stream));
    if (b->d_grids) cudaFree(b->d_grids);
    if (b->d_pre) cudaFree(b->d_pre);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->h_grids) cudaFreeHost(b->h_grids);
    if (b->h_pre) cudaFreeHost(b->h_pre);
    if (b->h_counters) cudaFreeHost(b->h_counters);
    b->d_grids = nullptr; b->d_pre = nullptr; b->d_counters = nullptr;
    b->h_grids = nullptr; b->h_pre = nullptr; b->h_counters = nullptr;
    SBP_CUDA(cudaMalloc(&b->d_grids, sizeof(sbp::BatchGrid) * cap));
    SBP_CUDA(cudaMalloc(&b->d_pre, sizeof(int) * 4 * (cap + 1)));
    SBP_CUDA(cudaMalloc(&b->d_counters, sizeof(long long) * cap));
    if (b->d_sched) cudaFree(b->d_sched);
    b->d_sched = nullptr;
    SBP_CUDA(cudaMalloc(&b->d_sched, sizeof(unsigned) * (2 * cap + 2)));
    SBP_CUDA(cudaMemsetAsync(b->d_sched, 0, sizeof(unsigned) * (2 * cap + 2), b->stream));
    SBP_CUDA(cudaHostAlloc((void **)&b->h_grids, sizeof(sbp::BatchGrid) * cap, cudaHostAllocDefault));
    SBP_CUDA(cudaHostAlloc((void **)&b->h_pre, sizeof(int) * 4 * (cap + 1), cudaHostAllocDefault));
    SBP_CUDA(cudaHostAlloc((void **)&b->h_counters, sizeof(long long) * cap, cudaHostAllocDefault));
    if (!b->staged) SBP_CUDA(cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming));
    b->cap = cap;
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    return SBP_OK;
}

// Upload every member's parameters, prefix tables and step counters.
constexpr int kBatchDepth = 64;   // z-planes per CTA of the batched one-pass step

int batch_rebuild(sbp_batch *b)
{
    const int n = (int)b->m.size();
    int rc = batch_reserve(b, std::max(n, 1));
    if (rc) return rc;
    // the previous upload must have left the pinned staging buffers
    SBP_CUDA(cudaEventSynchronize(b->staged));
    sbp::BatchGrid *hg = b->h_grids;
    int *pre = b->h_pre;
    long long *cnt = b->h_counters;
    std::memset(pre, 0, sizeof(int) * 4 * (b->cap + 1));
    int *pf = pre, *ph = pre + (b->cap + 1), *pe = pre + 2 * (b->cap + 1), *pi = pre + 3 * (b->cap + 1);
    // 16-row tiles (one 512-thread CTA per SM, which leaves room for the band
    // kernels beside it) when every member has a full one, and the per-step
    // path runs; else 8 rows (the persistent kernel always runs 8)
    int rows = b->persistent ? sbp::kFTY : 16;
    if (const char *env = std::getenv("SBP_FUSED_ROWS"))
        if (std::atoi(env) == 8) rows = sbp::kFTY;
    for (int g = 0; g < n; g++)
        if (b->m[g].s->n[1] - 5 < 15) rows = sbp::kFTY;
    b->rows = rows;
    for (int g = 0; g < n; g++) {
        sbp_sim *s = b->m[g].s;
        sbp::BatchGrid &G = hg[g];
        std::memset(static_cast<void *>(&G), 0, sizeof(G));
        // every member runs the batch's tile: 64 columns and the batch's height
        // (its TMA boxes are re-encoded when that differs from the member's own)
        if ((s->fused_rows != rows || s->fused_width != sbp::kFTX) &&
            (rc = set_tile(s, sbp::kFTX, rows, s->fused_kchunk)))
            return rc;
        for (int c = 0; c < 2; c++) {
            G.maps[c] = s->maps[c];
            if ((rc = make_fused_params(s, c, G.fp[c]))) return rc;
            if ((rc = make_params<float>(s, G.ph[c], c, c))) return rc;
            if ((rc = make_params<float>(s, G.pe[c], c, c ^ 1))) return rc;
            for (int f = 0; f < 3; f++) {
                G.hout[c][f] = static_cast<float *>(s->set[c ^ 1][3 + f]);
                G.eout[c][f] = static_cast<float *>(s->set[c ^ 1][f]);
            }
        }
        G.bh = s->band_hb;
        G.be = s->band_eb;
        G.counter = b->d_counters + g;
        G.target = b->m[g].target;
        G.cstart = s->step;
        G.probe_base = s->probe_base;
        G.cur0 = s->cur;
        // In a batch the other grids supply the parallelism that a lone grid
        // gets from many shallow z-blocks, so members run deep blocks (fewer
        // halo planes re-read, fewer pipeline fills): at least kBatchDepth.
        const int depth = std::max(s->fused_kchunk, kBatchDepth);
        G.fp[0].kchunk = G.fp[1].kchunk = depth;
        G.tiles[0] = s->fused_grid.x; G.tiles[1] = s->fused_grid.y;
        G.tiles[2] = (s->n[2] - 5 + depth - 1) / depth;
        cnt[g] = s->step;
        const long long nfg = (long long)G.tiles[0] * G.tiles[1] * G.tiles[2];
        const long long nhg = G.bh.ctas;
        const long long neg = G.be.ctas;
        if ((long long)pf[g] + nfg > INT32_MAX || (long long)ph[g] + nhg > INT32_MAX || (long long)pe[g] + neg > INT32_MAX)
            return SBP_ECAPACITY;
        pf[g + 1] = pf[g] + (int)nfg;
        ph[g + 1] = ph[g] + (int)nhg;
        pe[g + 1] = pe[g] + (int)neg;
        pi[g + 1] = pi[g] + sbp::band_items((int)nhg) + (int)nfg + sbp::band_items((int)neg);
    }
    b->nf = pf[n]; b->nh = ph[n]; b->ne = pe[n]; b->ni = pi[n];
    if (n > 0) {
        // stream-ordered behind the chunks already queued, which read the old tables
        SBP_CUDA(cudaMemcpyAsync(b->d_grids, hg, sizeof(sbp::BatchGrid) * n, cudaMemcpyHostToDevice, b->stream));
        SBP_CUDA(cudaMemcpyAsync(b->d_pre, pre, sizeof(int) * 4 * (b->cap + 1), cudaMemcpyHostToDevice, b->stream));
        SBP_CUDA(cudaMemcpyAsync(b->d_counters, cnt, sizeof(long long) * n, cudaMemcpyHostToDevice, b->stream));
        SBP_CUDA(cudaEventRecord(b->staged, b->stream));
    }
    b->gstale = true;                   // the graph is re-recorded and updated in place at the next chunk
    b->dirty = false;
    return SBP_OK;
}

// K steps of every member: offsets 0..K-1, then the counters advance by K.
int batch_launch_chunk(sbp_batch *b, long long K)
{
    const int n = (int)b->m.size();
    const int *pf = b->d_pre, *ph = b->d_pre + (b->cap + 1), *pe = b->d_pre + 2 * (b->cap + 1);
    if (b->persistent) {
        // one launch for the whole chunk: CTAs take (step, item) tickets in
        // order, items wait only for their own grid's previous step (see
        // persistent_batched); the counters start at zero
        const long long total = b->ni;
        if (total > 0 && K > 0) {
            if (total * K >= (1ll << 32) - 1) return SBP_ECAPACITY;
            SBP_CUDA(cudaMemsetAsync(b->d_sched, 0, sizeof(unsigned) * (2 * n + 1), b->stream));
            sbp::Persist P;
            P.ticket = b->d_sched;
            P.done = b->d_sched + 1;
            P.error_flag = reinterpret_cast<int *>(b->d_sched + 2 * b->cap + 1);
            P.wait_limit = 1u << 24;
            P.K = (int)K;
            P.n = n;
            P.cap = b->cap;
            P.total = (int)total;
            const long long grid = std::min<long long>(b->resident, total * K);
            sbp::persistent_batched<<<(unsigned)grid, sbp::kFTY * 32, sbp::kFusedSmem, b->stream>>>(
                b->d_grids, b->d_pre, b->d_pre + 3 * (b->cap + 1), P);
            SBP_CUDA(cudaGetLastError());
        }
    } else {
        // per step: the one-pass interior step on the batch stream, band H then
        // band E beside it on the side stream (band E reads only band H's output,
        // which includes the first interior H layer), joined before the next step
        for (long long o = 0; o < K; o++) {
            SBP_CUDA(cudaEventRecord(b->ev_fork, b->stream));
            if (b->nf > 0 && b->rows == 16)
                sbp::fused_batched<16><<<b->nf, 16 * 32, sbp::FusedGeom<float, 16>::kSmem, b->stream>>>(
                    b->d_grids, pf, n, (int)o);
            else if (b->nf > 0)
                sbp::fused_batched<8><<<b->nf, 8 * 32, sbp::FusedGeom<float, 8>::kSmem, b->stream>>>(
                    b->d_grids, pf, n, (int)o);
            SBP_CUDA(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
            if (b->nh > 0) sbp::band_h_batched<<<b->nh, 256, 0, b->side>>>(b->d_grids, ph, n, (int)o);
            if (b->ne > 0) sbp::band_e_batched<<<b->ne, 256, 0, b->side>>>(b->d_grids, pe, n, (int)o);
            SBP_CUDA(cudaEventRecord(b->ev_join, b->side));
            SBP_CUDA(cudaStreamWaitEvent(b->stream, b->ev_join, 0));
        }
    }
    sbp::batch_advance<<<(n + 127) / 128, 128, 0, b->stream>>>(b->d_grids, n, K);
    SBP_CUDA(cudaGetLastError());
    return SBP_OK;
}

// The energy monitor of a batch member: W at the member's current step into
// its series when the step is a multiple of energy_every (the steps inside a
// chunk are not sampled), behind the chunk on the batch's stream, and a copy
// of the sample to the member's host mirror if it has one.
int batch_sample_energy(sbp_batch *b, sbp_batch::Member &m)
{
    sbp_sim *s = m.s;
    if (s->energy_every <= 0 || s->step % s->energy_every) return SBP_OK;
    const long long idx = s->step / s->energy_every;
    if (idx >= s->eseries_cap) return SBP_ECAPACITY;
    int rc = energy_into(s, s->partials, s->eseries + idx);
    if (rc) return rc;
    s->eseries_count = std::max(s->eseries_count, idx + 1);
    if (m.mirror)
        SBP_CUDA(cudaMemcpyAsync(m.mirror, s->eseries + idx, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    return SBP_OK;
}

}  // namespace

namespace sbp {

// A dense (e0, e1, e2) field into the padded layout (row pitch sy, plane pitch
// sz) and back: host copies go through a contiguous staging array, so the DMA
// moves one block instead of e1 * e2 short rows.
template <typename T>
__global__ void put_field(const T *__restrict__ src, int e0, int e1, int e2, T *__restrict__ dst, long long sy,
                          long long sz)
{
    const long long total = (long long)e0 * e1 * e2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % e0);
        const int j = (int)((q / e0) % e1);
        const int k = (int)(q / ((long long)e0 * e1));
        dst[(long long)k * sz + (long long)j * sy + i] = src[q];
    }
}
template <typename T>
__global__ void get_field(const T *__restrict__ src, int e0, int e1, int e2, long long sy, long long sz,
                          T *__restrict__ dst)
{
    const long long total = (long long)e0 * e1 * e2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % e0);
        const int j = (int)((q / e0) % e1);
        const int k = (int)(q / ((long long)e0 * e1));
        dst[q] = src[(long long)k * sz + (long long)j * sy + i];
    }
}

}  // namespace sbp

extern "C" {

size_t sbp_workspace_bytes(const sbp_grid_desc *desc)
{
    if (!desc_valid(desc)) return 0;
    return make_layout(desc).total;
}

int sbp_create(const sbp_grid_desc *desc, void *cuda_stream, sbp_sim **out)
{
    return create_common(desc, cuda_stream, nullptr, 0, true, out);
}

int sbp_create_in(const sbp_grid_desc *desc, void *cuda_stream, void *dev_workspace, size_t bytes, sbp_sim **out)
{
    return create_common(desc, cuda_stream, dev_workspace, bytes, false, out);
}

int sbp_connect(sbp_sim *a, int fa, sbp_sim *b, int fb)
{
    if (!a || !b || fa < 0 || fa > 5 || fb < 0 || fb > 5) return SBP_EINVAL;
    if (a->fdtd || b->fdtd) return SBP_EINVAL;
    if (a->prec != b->prec || a->stream != b->stream) return SBP_EINVAL;
    const int ax = fa / 2;
    if (fb / 2 != ax || (fa % 2) == (fb % 2)) return SBP_ENOTCONFORMING;
    for (int t = 0; t < 3; t++) {
        if (t == ax) continue;
        if (a->n[t] != b->n[t] || a->h[t] != b->h[t]) return SBP_ENOTCONFORMING;
    }
    if (a->dt != b->dt) return SBP_ENOTCONFORMING;
    if (a->fscale[0] != b->fscale[0] || a->fscale[1] != b->fscale[1]) return SBP_EINVAL;
    a->face[fa] = SBP_INTERFACE; a->nbr[fa] = b; a->nbr_face[fa] = fb;
    b->face[fb] = SBP_INTERFACE; b->nbr[fb] = a; b->nbr_face[fb] = fa;
    a->nbr2[fa] = nullptr; a->nbr_w[fa][0] = 1.0; a->nbr_w[fa][1] = 0.0;
    b->nbr2[fb] = nullptr; b->nbr_w[fb][0] = 1.0; b->nbr_w[fb][1] = 0.0;
    return SBP_OK;
}

int sbp_connect_phase(sbp_sim *re, sbp_sim *im, int axis, double alpha)
{
    if (!re || !im || re == im || axis < 0 || axis > 2 || !std::isfinite(alpha)) return SBP_EINVAL;
    if (re->fdtd || im->fdtd) return SBP_EINVAL;
    if (re->prec != im->prec || re->stream != im->stream || re->dt != im->dt) return SBP_EINVAL;
    if (re->fscale[0] != im->fscale[0] || re->fscale[1] != im->fscale[1]) return SBP_EINVAL;
    for (int t = 0; t < 3; t++)
        if (re->n[t] != im->n[t] || re->h[t] != im->h[t]) return SBP_ENOTCONFORMING;
    // the field one period up is e^{-j alpha} times the field here: a high face
    // compares with e^{-j alpha} (low face), a low face with e^{+j alpha} (high face)
    const double c = std::cos(alpha), sn = std::sin(alpha);
    const int lo = 2 * axis, hi = 2 * axis + 1;
    sbp_sim *own[2] = {re, im}, *other[2] = {im, re};
    const double wb_hi[2] = {+sn, -sn}, wb_lo[2] = {-sn, +sn};
    for (int q = 0; q < 2; q++) {
        sbp_sim *s = own[q];
        s->face[lo] = SBP_INTERFACE; s->face[hi] = SBP_INTERFACE;
        s->nbr[hi] = s; s->nbr_face[hi] = lo; s->nbr2[hi] = other[q];
        s->nbr_w[hi][0] = c; s->nbr_w[hi][1] = wb_hi[q];
        s->nbr[lo] = s; s->nbr_face[lo] = hi; s->nbr2[lo] = other[q];
        s->nbr_w[lo][0] = c; s->nbr_w[lo][1] = wb_lo[q];
    }
    return SBP_OK;
}

int sbp_set_field(sbp_sim *s, int comp, const void *src, int is_device)
{
    int e[3];
    if (!s || !src || extents_of(s, comp, e)) return SBP_EINVAL;
    DeviceGuard dg(s->device);
    if (s->prec == SBP_FP32_FP16STORE) {
        // FP32 values in; stored as value / scale in FP16
        const size_t bytes = (size_t)e[0] * e[1] * e[2] * sizeof(float);
        const float *d_src = static_cast<const float *>(src);
        float *tmp = nullptr;
        if (!is_device) {
            SBP_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&tmp), bytes, s->stream));
            SBP_CUDA(cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, s->stream));
            d_src = tmp;
        }
        sbp::put_field_h<<<1024, 256, 0, s->stream>>>(d_src, e[0], e[1], e[2], static_cast<__half *>(s->set[s->cur][comp]),
                                                       s->sy, s->sz, (float)(1.0 / s->fscale[comp >= 3]));
        SBP_CUDA(cudaGetLastError());
        if (tmp) SBP_CUDA(cudaFreeAsync(tmp, s->stream));
        if (!is_device) SBP_CUDA(cudaStreamSynchronize(s->stream));
        return SBP_OK;
    }
    if (!is_device && s->fused_ok) {
        // host values: one contiguous copy into the spare set's array of this
        // component (dead between steps: the next step overwrites it), then a
        // scatter into the padded layout
        const size_t bytes = (size_t)e[0] * e[1] * e[2] * s->esize;
        void *stage = s->set[s->cur ^ 1][comp];
        SBP_CUDA(cudaMemcpyAsync(stage, src, bytes, cudaMemcpyHostToDevice, s->stream));
        if (s->esize == 8)
            sbp::put_field<double><<<1024, 256, 0, s->stream>>>(static_cast<const double *>(stage), e[0], e[1], e[2],
                                                               static_cast<double *>(s->set[s->cur][comp]), s->sy, s->sz);
        else
            sbp::put_field<float><<<1024, 256, 0, s->stream>>>(static_cast<const float *>(stage), e[0], e[1], e[2],
                                                              static_cast<float *>(s->set[s->cur][comp]), s->sy, s->sz);
        SBP_CUDA(cudaGetLastError());
        SBP_CUDA(cudaStreamSynchronize(s->stream));
        return SBP_OK;
    }
    cudaMemcpy3DParms m = {};
    m.srcPtr = make_cudaPitchedPtr(const_cast<void *>(src), e[0] * s->esize, e[0] * s->esize, e[1]);
    m.dstPtr = make_cudaPitchedPtr(s->set[s->cur][comp], s->sy * s->esize, e[0] * s->esize, s->n[1] + 2);
    m.extent = make_cudaExtent(e[0] * s->esize, e[1], e[2]);
    m.kind = cudaMemcpyDefault;
    SBP_CUDA(cudaMemcpy3DAsync(&m, s->stream));
    if (!is_device) SBP_CUDA(cudaStreamSynchronize(s->stream));
    return SBP_OK;
}

int sbp_get_field(sbp_sim *s, int comp, void *dst, int to_device)
{
    int e[3];
    if (!s || !dst || extents_of(s, comp, e)) return SBP_EINVAL;
    DeviceGuard dg(s->device);
    if (s->prec == SBP_FP32_FP16STORE) {
        // stored FP16 values times the field's scale, out as FP32
        const size_t bytes = (size_t)e[0] * e[1] * e[2] * sizeof(float);
        float *d_dst = static_cast<float *>(dst);
        if (!to_device) SBP_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&d_dst), bytes, s->stream));
        sbp::get_field_h<<<1024, 256, 0, s->stream>>>(static_cast<const __half *>(s->set[s->cur][comp]), e[0], e[1], e[2],
                                                       s->sy, s->sz, (float)s->fscale[comp >= 3], d_dst);
        SBP_CUDA(cudaGetLastError());
        if (!to_device) {
            SBP_CUDA(cudaMemcpyAsync(dst, d_dst, bytes, cudaMemcpyDeviceToHost, s->stream));
            SBP_CUDA(cudaFreeAsync(d_dst, s->stream));
            SBP_CUDA(cudaStreamSynchronize(s->stream));
            return check_error_flag(s);
        }
        return SBP_OK;
    }
    if (!to_device && s->fused_ok) {
        // gather into the spare set's array (dead between steps), then one
        // contiguous copy to the host
        const size_t bytes = (size_t)e[0] * e[1] * e[2] * s->esize;
        void *stage = s->set[s->cur ^ 1][comp];
        if (s->esize == 8)
            sbp::get_field<double><<<1024, 256, 0, s->stream>>>(static_cast<const double *>(s->set[s->cur][comp]), e[0],
                                                               e[1], e[2], s->sy, s->sz, static_cast<double *>(stage));
        else
            sbp::get_field<float><<<1024, 256, 0, s->stream>>>(static_cast<const float *>(s->set[s->cur][comp]), e[0],
                                                              e[1], e[2], s->sy, s->sz, static_cast<float *>(stage));
        SBP_CUDA(cudaGetLastError());
        SBP_CUDA(cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyDeviceToHost, s->stream));
        SBP_CUDA(cudaStreamSynchronize(s->stream));
        return check_error_flag(s);
    }
    cudaMemcpy3DParms m = {};
    m.srcPtr = make_cudaPitchedPtr(s->set[s->cur][comp], s->sy * s->esize, e[0] * s->esize, s->n[1] + 2);
    m.dstPtr = make_cudaPitchedPtr(dst, e[0] * s->esize, e[0] * s->esize, e[1]);
    m.extent = make_cudaExtent(e[0] * s->esize, e[1], e[2]);
    m.kind = cudaMemcpyDefault;
    SBP_CUDA(cudaMemcpy3DAsync(&m, s->stream));
    if (!to_device) {
        SBP_CUDA(cudaStreamSynchronize(s->stream));
        return check_error_flag(s);
    }
    return SBP_OK;
}

int sbp_add_source(sbp_sim *s, int comp, int i, int j, int k, int waveform, double amp, double tw, double t0, double f)
{
    int e[3];
    if (!s || comp < 0 || comp > 2 || extents_of(s, comp, e)) return SBP_EINVAL;
    if ((int)s->src.size() >= sbp::kMaxSources) return SBP_ECAPACITY;
    if (waveform < SBP_GAUSS || waveform > SBP_MOD_GAUSS || !(tw > 0)) return SBP_EINVAL;
    const int idx[3] = {i, j, k};
    for (int a = 0; a < 3; a++)
        if (idx[a] < -1 || idx[a] >= e[a]) return SBP_EINVAL;
    sbp::Src q;
    q.comp = comp; q.i = i; q.j = j; q.k = k; q.wf = waveform;
    q.amp = amp; q.tw = tw; q.t0 = t0; q.f = f;
    s->src.push_back(q);
    return (int)s->src.size() - 1;
}

int sbp_add_probe(sbp_sim *s, int comp, int i, int j, int k, int *probe_id)
{
    int e[3];
    if (!s || extents_of(s, comp, e)) return SBP_EINVAL;
    if ((int)s->prb.size() >= sbp::kMaxProbes) return SBP_ECAPACITY;
    const int idx[3] = {i, j, k};
    for (int a = 0; a < 3; a++)
        if (idx[a] < 0 || idx[a] >= e[a]) return SBP_EINVAL;
    if (s->probe_buf) return SBP_ESTATE;    // add probes before reserving their buffer
    sbp::Prb q;
    q.comp = comp; q.i = i; q.j = j; q.k = k;
    s->prb.push_back(q);
    if (probe_id) *probe_id = (int)s->prb.size() - 1;
    return SBP_OK;
}

int sbp_reserve_probes(sbp_sim *s, int64_t nsteps)
{
    if (!s || nsteps < 0) return SBP_EINVAL;
    DeviceGuard dg(s->device);
    SBP_CUDA(cudaStreamSynchronize(s->stream));
    if (s->probe_buf) { cudaFree(s->probe_buf); s->probe_buf = nullptr; }
    s->probe_cap = 0;
    const size_t np = std::max<size_t>(1, s->prb.size());
    if (nsteps > 0) {
        SBP_CUDA(cudaMalloc(&s->probe_buf, np * nsteps * s->psize));
        SBP_CUDA(cudaMemsetAsync(s->probe_buf, 0, np * nsteps * s->psize, s->stream));
        s->probe_cap = nsteps;
    }
    s->probe_base = s->step;
    return SBP_OK;
}

int sbp_step(sbp_sim *s, int64_t nsteps)
{
    if (!s) return SBP_EINVAL;
    sbp_sim *one[1] = {s};
    return step_group(one, 1, nsteps);
}

int sbp_step_group(sbp_sim **sims, int nsims, int64_t nsteps)
{
    return step_group(sims, nsims, nsteps);
}

int sbp_half_step_h(sbp_sim **sims, int nsims)
{
    int rc = check_group(sims, nsims);
    if (rc) return rc;
    for (int q = 0; q < nsims; q++)
        if (sims[q]->fdtd) return SBP_ESTATE;
    DeviceGuard dg(sims[0]->device);
    return half_h(sims, nsims);
}

int sbp_half_step_e(sbp_sim **sims, int nsims)
{
    int rc = check_group(sims, nsims);
    if (rc) return rc;
    for (int q = 0; q < nsims; q++)
        if (sims[q]->fdtd) return SBP_ESTATE;
    DeviceGuard dg(sims[0]->device);
    return half_e(sims, nsims);
}

int sbp_step_timed(sbp_sim *s, int64_t nsteps, double *avg_ms, int64_t *launches, int n_out)
{
    if (!s || nsteps < 0) return SBP_EINVAL;
    sbp_sim *one[1] = {s};
    int rc = check_group(one, 1);
    if (rc) return rc;
    DeviceGuard dg(s->device);
    if (s->energy_every > 0) {
        rc = ensure_series(s, (s->step + nsteps) / s->energy_every + 1);
        if (rc) return rc;
    }
    return step_timed(s, nsteps, avg_ms, launches, n_out);
}

int sbp_tile(const sbp_sim *s, int *rows, int *depth, int *width)
{
    if (!s) return SBP_EINVAL;
    if (!s->fused_ok) return SBP_ESTATE;
    if (rows) *rows = s->fused_rows;
    if (depth) *depth = s->fused_kchunk;
    if (width) *width = s->fused_width;
    return SBP_OK;
}

int sbp_autotune(sbp_sim *s, int trial_steps, int *chosen_depth, double *ms_per_step)
{
    if (!s || trial_steps < 1) return SBP_EINVAL;
    DeviceGuard dg(s->device);
    return autotune(s, trial_steps, chosen_depth, ms_per_step);
}

int sbp_get_probes(sbp_sim *s, double *out, int64_t cap, int64_t *nsamples)
{
    if (!s || cap < 0 || (!out && cap > 0)) return SBP_EINVAL;
    DeviceGuard dg(s->device);
    SBP_CUDA(cudaStreamSynchronize(s->stream));
    const long long rec = std::min<long long>(s->step - s->probe_base, s->probe_cap);
    if (nsamples) *nsamples = rec;
    const size_t np = s->prb.size();
    if (np == 0 || !s->probe_buf || cap == 0) return SBP_OK;
    std::vector<char> host(np * s->probe_cap * s->psize);
    SBP_CUDA(cudaMemcpy(host.data(), s->probe_buf, host.size(), cudaMemcpyDeviceToHost));
    const long long m = std::min<long long>(cap, s->probe_cap);
    for (size_t q = 0; q < np; q++)
        for (long long t = 0; t < m; t++) {
            const size_t src = q * s->probe_cap + t;
            out[q * cap + t] = s->psize == 8 ? reinterpret_cast<double *>(host.data())[src]
                                             : (double)reinterpret_cast<float *>(host.data())[src];
        }
    return SBP_OK;
}

int sbp_energy_group(sbp_sim **sims, int nsims, double *W)
{
    Trace trace("sbp_energy");
    if (!sims || nsims <= 0 || !W) return SBP_EINVAL;
    double total = 0.0;
    for (int q = 0; q < nsims; q++) {
        sbp_sim *s = sims[q];
        if (!s) return SBP_EINVAL;
        if (s->fdtd) return SBP_ESTATE;   // the energy of Eq. (16) is not the Yee scheme's
        DeviceGuard dg(s->device);
        int rc = launch_h_any(s, true, false);
        if (rc) return rc;
        rc = finalize_energy(s, s->escalar);
        if (rc) return rc;
        double v = 0.0;
        SBP_CUDA(cudaMemcpyAsync(&v, s->escalar, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        SBP_CUDA(cudaStreamSynchronize(s->stream));
        total += v;
    }
    *W = total;
    return SBP_OK;
}

int sbp_energy(sbp_sim *s, double *W)
{
    sbp_sim *one[1] = {s};
    return sbp_energy_group(one, 1, W);
}

int sbp_energy_noalloc(sbp_sim *s, double *W_dev)
{
    if (!s || !W_dev || (reinterpret_cast<uintptr_t>(W_dev) & 7)) return SBP_EINVAL;
    if (s->fdtd) return SBP_ESTATE;
    if (s->npartials > SBP_NOALLOC_MAX_PARTIALS) {
        std::fprintf(stderr, "sbp_energy_noalloc: grid needs %lld partial sums, limit %d\n",
                     s->npartials, SBP_NOALLOC_MAX_PARTIALS);
        return SBP_ECAPACITY;
    }
    // W_dev must be device memory of the simulation's device: a host pointer
    // or another GPU's memory would be written through an address the
    // kernel cannot use.
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, W_dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return SBP_EINVAL;
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != s->device)
        return SBP_EINVAL;
    DeviceGuard dg(s->device);
    return energy_into(s, s->noalloc_partials, W_dev);
}

int sbp_energy_series(sbp_sim *s, double *out, int64_t cap, int64_t *count)
{
    if (!s || cap < 0 || (!out && cap > 0)) return SBP_EINVAL;
    DeviceGuard dg(s->device);
    SBP_CUDA(cudaStreamSynchronize(s->stream));
    if (count) *count = s->eseries_count;
    if (s->eseries_count == 0) return SBP_OK;
    std::vector<double> host(s->eseries_count);
    SBP_CUDA(cudaMemcpy(host.data(), s->eseries, host.size() * sizeof(double), cudaMemcpyDeviceToHost));
    const long long m = std::min<long long>(cap, s->eseries_count);
    for (long long t = 0; t < m; t++) out[t] = host[t];
    for (double v : host)
        if (!std::isfinite(v) || v > 1.5 * host[0]) return SBP_EUNSTABLE;
    return SBP_OK;
}

int sbp_sync(sbp_sim *s)
{
    if (!s) return SBP_EINVAL;
    DeviceGuard dg(s->device);
    SBP_CUDA(cudaStreamSynchronize(s->stream));
    return check_error_flag(s);
}

// Checkpoint blob: header, the six stored fields of the current set (whole
// padded arrays, raw storage values), the probe samples, the energy series.
struct CkptHeader {
    char magic[8];
    int32_t version, precision;
    int32_t n[3], nprobes;
    int64_t step, probe_base, probe_cap, eseries_count;
    uint64_t field_elems, esize, psize;
};
constexpr char kCkptMagic[8] = {'S', 'B', 'P', 'C', 'K', 'P', 'T', '1'};

size_t ckpt_bytes(const sbp_sim *s)
{
    const size_t np = s->probe_buf ? s->prb.size() : 0;
    return sizeof(CkptHeader) + 6 * s->field_elems * s->esize + np * (size_t)s->probe_cap * s->psize +
           (size_t)s->eseries_count * sizeof(double);
}

size_t sbp_checkpoint_bytes(const sbp_sim *s) { return s ? ckpt_bytes(s) : 0; }

int sbp_save(sbp_sim *s, void *host, size_t bytes)
{
    Trace trace("sbp_save");
    if (!s || !host) return SBP_EINVAL;
    if (bytes < ckpt_bytes(s)) return SBP_ECAPACITY;
    DeviceGuard dg(s->device);
    SBP_CUDA(cudaStreamSynchronize(s->stream));
    int rc = check_error_flag(s);
    if (rc) return rc;
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.precision = s->prec;
    for (int a = 0; a < 3; a++) h.n[a] = s->n[a];
    h.nprobes = s->probe_buf ? (int32_t)s->prb.size() : 0;
    h.step = s->step;
    h.probe_base = s->probe_base;
    h.probe_cap = s->probe_buf ? s->probe_cap : 0;
    h.eseries_count = s->eseries_count;
    h.field_elems = s->field_elems;
    h.esize = s->esize;
    h.psize = s->psize;
    char *p = static_cast<char *>(host);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const size_t fb = s->field_elems * s->esize;
    for (int c = 0; c < 6; c++, p += fb) SBP_CUDA(cudaMemcpy(p, s->set[s->cur][c], fb, cudaMemcpyDeviceToHost));
    const size_t pb = (size_t)h.nprobes * (size_t)h.probe_cap * s->psize;
    if (pb) { SBP_CUDA(cudaMemcpy(p, s->probe_buf, pb, cudaMemcpyDeviceToHost)); p += pb; }
    if (h.eseries_count)
        SBP_CUDA(cudaMemcpy(p, s->eseries, h.eseries_count * sizeof(double), cudaMemcpyDeviceToHost));
    return SBP_OK;
}

int sbp_load(sbp_sim *s, const void *host, size_t bytes)
{
    Trace trace("sbp_load");
    if (!s || !host || bytes < sizeof(CkptHeader)) return SBP_EINVAL;
    CkptHeader h;
    std::memcpy(&h, host, sizeof(h));
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1 || h.precision != s->prec ||
        h.field_elems != s->field_elems || h.esize != s->esize || h.psize != s->psize)
        return SBP_EINVAL;
    for (int a = 0; a < 3; a++)
        if (h.n[a] != s->n[a]) return SBP_EINVAL;
    if (h.nprobes != 0 && h.nprobes != (int32_t)s->prb.size()) return SBP_EINVAL;
    const size_t fb = s->field_elems * s->esize;
    const size_t pb = (size_t)h.nprobes * (size_t)h.probe_cap * s->psize;
    if (bytes < sizeof(h) + 6 * fb + pb + (size_t)h.eseries_count * sizeof(double)) return SBP_ECAPACITY;
    DeviceGuard dg(s->device);
    int rc;
    if (h.nprobes && (!s->probe_buf || s->probe_cap != h.probe_cap)) {
        if ((rc = sbp_reserve_probes(s, h.probe_cap))) return rc;
    }
    if (h.eseries_count && (rc = ensure_series(s, h.eseries_count))) return rc;
    SBP_CUDA(cudaStreamSynchronize(s->stream));
    const char *p = static_cast<const char *>(host) + sizeof(h);
    for (int c = 0; c < 6; c++, p += fb) SBP_CUDA(cudaMemcpy(s->set[s->cur][c], p, fb, cudaMemcpyHostToDevice));
    if (pb) { SBP_CUDA(cudaMemcpy(s->probe_buf, p, pb, cudaMemcpyHostToDevice)); p += pb; }
    if (h.eseries_count) SBP_CUDA(cudaMemcpy(s->eseries, p, h.eseries_count * sizeof(double), cudaMemcpyHostToDevice));
    s->step = h.step;
    s->probe_base = h.probe_base;
    s->eseries_count = h.eseries_count;
    return SBP_OK;
}

double sbp_dt(const sbp_sim *s) { return s ? s->dt : 0.0; }
int64_t sbp_step_index(const sbp_sim *s) { return s ? s->step : -1; }

int sbp_destroy(sbp_sim *s)
{
    if (!s) return SBP_EINVAL;
    DeviceGuard dg(s->device);
    cudaStreamSynchronize(s->stream);
    for (int f = 0; f < 6; f++) {
        sbp_sim *nb = s->nbr[f];
        if (nb && nb != s && s->nbr_face[f] >= 0 && nb->nbr[s->nbr_face[f]] == s) nb->nbr[s->nbr_face[f]] = nullptr;
    }
    if (s->side) { cudaStreamSynchronize(s->side); cudaStreamDestroy(s->side); }
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->probe_buf) cudaFree(s->probe_buf);
    if (s->eseries) cudaFree(s->eseries);
    if (s->own_ws && s->workspace) cudaFree(s->workspace);
    delete s;
    return SBP_OK;
}

int sbp_batch_create(void *cuda_stream, int flags, sbp_batch **out)
{
    if (!out || (flags & ~(SBP_BATCH_GRAPHS | SBP_BATCH_PERSISTENT))) return SBP_EINVAL;
    sbp_batch *b = new (std::nothrow) sbp_batch();
    if (!b) return SBP_ENOMEM;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->use_graph = (flags & SBP_BATCH_GRAPHS) != 0;
    b->persistent = (flags & SBP_BATCH_PERSISTENT) != 0;
    cudaGetDevice(&b->device);
    int rc = set_fused_smem_attr();
    if (rc) { delete b; return rc; }
    // CTAs of the persistent kernel that fit on the device at once
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sbp::persistent_batched, sbp::kFTY * 32,
                                                      sbp::kFusedSmem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
        cudaHostAlloc((void **)&b->h_err, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        (void)cudaGetLastError();
        delete b;
        return SBP_ECUDA;
    }
    *b->h_err = 0;
    b->resident = std::max(1, per_sm * sms);
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        if (b->side) cudaStreamDestroy(b->side);
        if (b->ev_fork) cudaEventDestroy(b->ev_fork);
        if (b->ev_join) cudaEventDestroy(b->ev_join);
        delete b;
        return SBP_ECUDA;
    }
    *out = b;
    return SBP_OK;
}

int sbp_batch_add(sbp_batch *b, sbp_sim *s, int64_t nsteps)
{
    if (!b || !s || nsteps < 0) return SBP_EINVAL;
    if (!s->fused_ok || s->prec != SBP_FP32 || s->fdtd || s->stream != b->stream || s->device != b->device)
        return SBP_EINVAL;
    for (int f = 0; f < 6; f++)
        if (s->face[f] == SBP_INTERFACE) return SBP_EINVAL;
    for (auto &m : b->m)
        if (m.s == s) return SBP_ESTATE;
    DeviceGuard dg(b->device);
    if (s->energy_every > 0) {
        // room for every sample up to the target step, then the sample at the current step
        int rc = ensure_series(s, (s->step + nsteps) / s->energy_every + 1);
        if (rc) return rc;
    }
    b->m.push_back({s, s->step + nsteps, nullptr});
    b->dirty = true;
    return batch_sample_energy(b, b->m.back());
}

int sbp_batch_remove(sbp_batch *b, sbp_sim *s)
{
    if (!b || !s) return SBP_EINVAL;
    for (size_t g = 0; g < b->m.size(); g++)
        if (b->m[g].s == s) {
            b->m.erase(b->m.begin() + g);
            b->dirty = true;
            return SBP_OK;
        }
    return SBP_EINVAL;
}

int sbp_batch_remaining(const sbp_batch *b, const sbp_sim *s, int64_t *remaining)
{
    if (!b || !s || !remaining) return SBP_EINVAL;
    for (auto &m : b->m)
        if (m.s == s) {
            *remaining = m.target - s->step;
            return SBP_OK;
        }
    return SBP_EINVAL;
}

int sbp_batch_step(sbp_batch *b, int64_t nsteps)
{
    Trace trace("sbp_batch_step");
    if (!b || nsteps < 0) return SBP_EINVAL;
    DeviceGuard dg(b->device);
    // a wait of an earlier persistent launch gave up (the flag is copied out
    // behind every chunk)
    if (*static_cast<volatile int *>(b->h_err)) return SBP_ETIMEOUT;
    if (b->m.empty() || nsteps == 0) return SBP_OK;
    int rc = SBP_OK;
    if (b->dirty && (rc = batch_rebuild(b))) return rc;
    if (b->use_graph) {
        if (!b->gexec || b->gK != nsteps || b->gstale) {
            // record the chunk on the private stream (nothing executes during
            // capture), then launch the graph on the batch's stream, which may
            // be the legacy default stream that cannot itself be captured
            cudaGraph_t graph = nullptr;
            SBP_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
            cudaStream_t keep = b->stream;
            b->stream = b->cap_stream;
            rc = batch_launch_chunk(b, nsteps);
            b->stream = keep;
            cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
            if (rc || e != cudaSuccess) {
                (void)cudaGetLastError();
                if (graph) cudaGraphDestroy(graph);
                return rc ? rc : SBP_ECUDA;
            }
            // a membership change alters only launch sizes and parameters: update
            // the executable graph in place when the topology allows, else
            // instantiate it anew
            bool updated = false;
            if (b->gexec && b->gK == nsteps) {
                cudaGraphExecUpdateResultInfo info;
                updated = cudaGraphExecUpdate(b->gexec, graph, &info) == cudaSuccess;
                if (!updated) (void)cudaGetLastError();
            }
            if (!updated) {
                if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
                e = cudaGraphInstantiate(&b->gexec, graph, 0);
                if (e != cudaSuccess) {
                    (void)cudaGetLastError();
                    cudaGraphDestroy(graph);
                    b->gexec = nullptr;
                    return SBP_ECUDA;
                }
            }
            cudaGraphDestroy(graph);
            b->gK = nsteps;
            b->gstale = false;
        }
        SBP_CUDA(cudaGraphLaunch(b->gexec, b->stream));
    } else {
        if ((rc = batch_launch_chunk(b, nsteps))) return rc;
    }
    if (b->persistent)
        SBP_CUDA(cudaMemcpyAsync(b->h_err, b->d_sched + 2 * b->cap + 1, sizeof(int), cudaMemcpyDeviceToHost,
                                 b->stream));
    // host bookkeeping: every member took min(nsteps, remaining) steps; then
    // the energy monitor of the members that reached a sampling step
    for (auto &m : b->m) {
        const long long done = std::min<long long>(nsteps, std::max<long long>(0, m.target - m.s->step));
        m.s->step += done;
        m.s->cur ^= (int)(done & 1);
        if (done > 0 && (rc = batch_sample_energy(b, m))) return rc;
    }
    return SBP_OK;
}

int sbp_batch_size(const sbp_batch *b) { return b ? (int)b->m.size() : 0; }

int sbp_batch_destroy(sbp_batch *b)
{
    if (!b) return SBP_EINVAL;
    DeviceGuard dg(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->d_grids) cudaFree(b->d_grids);
    if (b->d_pre) cudaFree(b->d_pre);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->h_grids) cudaFreeHost(b->h_grids);
    if (b->h_pre) cudaFreeHost(b->h_pre);
    if (b->h_counters) cudaFreeHost(b->h_counters);
    if (b->d_sched) cudaFree(b->d_sched);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->staged) cudaEventDestroy(b->staged);
    delete b;
    return SBP_OK;
}

}  // extern "C"

#include "server.cuh"

extern "C" {

const char *sbp_strerror(int code)
{
    switch (code) {
    case SBP_OK: return "ok";
    case SBP_EINVAL: return "invalid argument";
    case SBP_ENOMEM: return "out of memory";
    case SBP_ECUDA: return "CUDA runtime error";
    case SBP_EUNSTABLE: return "energy monitor: growth or non-finite value";
    case SBP_ETIMEOUT: return "bounded device wait timed out";
    case SBP_ENOTCONFORMING: return "interface faces do not conform";
    case SBP_ESTATE: return "call not valid in the current state";
    case SBP_ECAPACITY: return "buffer too small";
    case SBP_EAGAIN: return "not finished yet";
    default: return "unknown error";
    }
}

}  // extern "C"
