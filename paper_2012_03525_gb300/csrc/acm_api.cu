// C ABI of libacm: handle life cycle, parameter validation, field transfer,
// time stepping (with CUDA-graph replay) and diagnostics.  All arithmetic of
// the scheme runs in the kernels of acm_step2d.cu / acm_step3d.cu /
// acm_reduce.cu; this file only marshals.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "acm_internal.h"

using namespace acm;

namespace {
// NVTX range over one API call (visible in Nsight timelines; no cost when no
// tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

struct acm_handle {
    int nruns = 0, dim = 2, prec = ACM_FP64, two_phase = 0, any_wall = 0;
    int scheme = ACM_SCHEME_SMAMES;
    std::vector<acm_params> params;
    std::vector<RunDesc> runs;
    std::vector<long long> npoints;   // nodes per run
    std::vector<char> have_fields;
    RunDesc *druns = nullptr;
    int4 *dwork = nullptr;
    int nwork = 0;
    int4 *dline = nullptr;            // 2D line-marching work list (empty if it does not apply)
    int nline = 0;
    bool line_gen = false;            // some run has rho0 != 1 or a body force
    size_t pool = 0;                  // elements per field pool
    void *buf[2][NFIELD] = {};
    int cur = 0;
    int64_t steps = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool own_fields = true;           // false: acm_create_ext (caller-owned buffers)
    unsigned *derr = nullptr;
    unsigned sticky = 0;
    double *dpartials = nullptr;
    int red_blocks = 0;
    double *dout = nullptr;
    double *dstage = nullptr;
    std::vector<CUtensorMap> maps;  // 3D: [buffer][run][field]
    bool maps_ok = false;
    bool halo = false;              // 3D sub-domains (ACM_BC_HALO z faces)
    // sub-domains step concurrently: slab r > 0 runs on side[r - 1], forked
    // from and joined back into `stream` with events
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;    // [0] fork, [r] join of slab r
    void *scratch[3] = {};          // 3D two-phase: mu, phi*, Delta rho
    cudaGraphExec_t gexec = nullptr;
    Tuning tune;
    std::string err;
    int device = 0, sms = 0;
    size_t esize() const { return prec == ACM_FP64 ? sizeof(double) : sizeof(float); }
};

namespace {

thread_local std::string g_thread_err;

acm_status fail(acm_handle *h, acm_status st, const std::string &msg)
{
    if (h) h->err = msg;
    else g_thread_err = msg;
    return st;
}

acm_status cuda_fail(acm_handle *h, cudaError_t e, const char *what)
{
    // a failed runtime call stays the thread's last error; clear it, so that a
    // non-sticky failure (an allocation that did not fit) is not reported
    // again by the next launch on a context that is still usable
    (void)cudaGetLastError();
    return fail(h, e == cudaErrorMemoryAllocation ? ACM_ENOMEM : ACM_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                              \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

bool valid_bc(int b)
{
    return b == ACM_BC_PERIODIC || b == ACM_BC_WALL || b == ACM_BC_LID || b == ACM_BC_HALO ||
           b == ACM_BC_SYMMETRY;
}

acm_status validate(const acm_params &p, std::string &why)
{
    auto bad = [&](const char *m) {
        why = m;
        return ACM_EINVAL;
    };
    if (p.dim != 2 && p.dim != 3) return bad("dim must be 2 or 3");
    if (p.nx < 1 || p.ny < 1 || (p.dim == 3 && p.nz < 1)) return bad("grid sizes must be >= 1");
    if (p.dim == 2 && p.nz != 1) return bad("nz must be 1 in 2D");
    if (!(p.dt > 0) || !std::isfinite(p.dt)) return bad("dt must be > 0");
    if (!(p.nu >= 0) || !std::isfinite(p.nu)) return bad("nu must be >= 0");
    if (!std::isfinite(p.rho0) || !(p.rho0 > 0)) return bad("rho0 must be > 0");
    if (p.precision != ACM_FP64 && p.precision != ACM_FP32_DEV) return bad("bad precision");
    if (p.sat_mask < 0 || p.sat_mask > 3) return bad("sat_mask must be 0..3");
    const int n[3] = {p.nx, p.ny, p.nz};
    for (int d = 0; d < 3; ++d) {
        const int lo = p.bc[2 * d], hi = p.bc[2 * d + 1];
        if (d >= p.dim) continue;
        if (!valid_bc(lo) || !valid_bc(hi)) return bad("unknown boundary kind");
        if ((lo == ACM_BC_HALO) != (hi == ACM_BC_HALO))
            return bad("ACM_BC_HALO must be on both faces of an axis");
        if (lo == ACM_BC_HALO) {
            if (p.dim != 3 || d != 2) return bad("ACM_BC_HALO is for the z faces of 3D grids");
            if (n[d] < 2) return bad("sub-domains need nz >= 2");
            continue;
        }
        if ((lo == ACM_BC_SYMMETRY) != (hi == ACM_BC_SYMMETRY))
            return bad("a symmetry face must be paired with a symmetry face");
        if (lo == ACM_BC_SYMMETRY) {
            if (p.dim != 3 || !p.two_phase || d == 2)
                return bad("symmetry planes are for the x and y faces of 3D two-phase runs");
            if (n[d] < 3) return bad("symmetry planes need >= 3 nodes across");
            continue;
        }
        if ((lo == ACM_BC_PERIODIC) != (hi == ACM_BC_PERIODIC))
            return bad("a periodic face must be paired with a periodic face");
        if (lo != ACM_BC_PERIODIC && n[d] < 4) return bad("walls need >= 4 nodes across");
    }
    if (p.dim == 3) {
        for (int f = 0; f < 4; ++f)
            if (p.bc[f] != ACM_BC_PERIODIC && p.bc[f] != ACM_BC_SYMMETRY)
                return bad("3D grids need periodic or symmetry x and y faces");
        const int zb = p.bc[4];
        if (zb == ACM_BC_LID) return bad("3D grids have no lid faces");
        if (zb == ACM_BC_WALL && !p.two_phase)
            return bad("3D z walls are supported for two-phase runs only");
        if (zb == ACM_BC_HALO && p.two_phase) return bad("3D sub-domains are single-phase only");
        if (p.nx < 2 || p.ny < 2) return bad("3D grids need nx, ny >= 2");
    }
    if (p.scheme != ACM_SCHEME_SMAMES && p.scheme != ACM_SCHEME_MAMES) return bad("unknown scheme");
    if (p.scheme == ACM_SCHEME_MAMES) {
        if (p.dim != 2 || p.two_phase) return bad("the MAMEs scheme is 2D single-phase only");
        for (int f = 0; f < 4; ++f)
            if (p.bc[f] != ACM_BC_PERIODIC) return bad("the MAMEs scheme needs periodic faces");
        if (p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0)
            return bad("the MAMEs scheme takes no body force");
    }
    if (p.two_phase) {
        if (!(p.W > 0) || !(p.sigma >= 0) || !(p.M >= 0)) return bad("bad sigma/W/M");
        if (!std::isfinite(p.theta_deg)) return bad("non-finite contact angle");
    }
    if (!std::isfinite(p.rho_ratio) || p.rho_ratio < 0) return bad("rho_ratio must be >= 0");
    if (p.rho_ratio > 0 && !p.two_phase) return bad("rho_ratio needs a two-phase run");
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(p.g[d]) || !std::isfinite(p.lid_u[d])) return bad("non-finite g/lid");
    return ACM_OK;
}

RunDesc describe(const acm_params &p)
{
    RunDesc r;
    std::memset(&r, 0, sizeof(r));
    r.nx = p.nx;
    r.ny = p.ny;
    r.nz = p.dim == 3 ? p.nz : 1;
    for (int f = 0; f < 6; ++f) r.bc[f] = p.bc[f];
    r.rho0 = p.rho0;
    r.dt = p.dt;
    r.cs2 = 1.0 / (3.0 * p.dt * p.dt);
    r.nu = p.nu;
    for (int d = 0; d < 3; ++d) {
        r.g[d] = p.g[d];
        r.lid[d] = p.lid_u[d];
    }
    r.two_phase = p.two_phase;
    r.a = 3.0 * p.sigma / (4.0 * p.W);
    r.kappa = 3.0 * p.sigma * p.W / 8.0;
    r.M = p.M;
    r.sat_c = p.sat_mask & 1;
    r.sat_m = (p.sat_mask >> 1) & 1;
    double c[NCOEF];
    c[C_RHO0] = r.rho0;
    c[C_DT] = r.dt;
    c[C_CS2] = r.cs2;
    c[C_NU] = r.nu;
    c[C_SATC] = r.sat_c ? 0.5 * r.cs2 * r.dt * r.dt : 0.0;
    c[C_SATM] = r.sat_m ? r.nu + 0.5 * r.cs2 * r.dt : 0.0;
    c[C_NUDT] = r.nu * r.dt;
    c[C_GX] = r.g[0];
    c[C_GY] = r.g[1];
    c[C_GZ] = r.g[2];
    c[C_LIDX] = r.lid[0];
    c[C_LIDY] = r.lid[1];
    c[C_LIDZ] = r.lid[2];
    c[C_A] = r.a;
    c[C_KAPPA] = r.kappa;
    c[C_M] = r.M;
    c[C_WET] = 2.0 * (2.0 / p.W) * std::cos(p.theta_deg * 3.14159265358979323846 / 180.0);
    if (p.two_phase && p.rho_ratio > 0) {
        const double beta = 2.0 * (p.rho_ratio - 1.0) / (p.rho_ratio + 1.0);
        c[C_BQA] = 0.5 * beta;
        c[C_BQB] = 0.5 * beta;
    } else {
        c[C_BQA] = 1.0;
        c[C_BQB] = 0.0;
    }
    for (int k = 0; k < NCOEF; ++k) {
        r.cd[k] = c[k];
        r.cf[k] = (float)c[k];
    }
    r.zg = (p.dim == 3 && p.bc[4] == ACM_BC_HALO) ? 2 : 0;
    if (p.dim == 3) {
        r.pad = T3PAD;
        r.px = ((p.nx + 2 * T3PAD + 7) / 8) * 8;
        r.py = p.ny + 2 * T3PAD;
    } else {
        r.pad = 0;
        r.px = p.nx;
        r.py = p.ny;
    }
    return r;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

acm_status build_maps(acm_handle *h)
{
    h->maps_ok = false;
    if (h->dim != 3) return ACM_OK;
    auto fn = encode_fn();
    if (!fn) return fail(h, ACM_ECUDA, "cuTensorMapEncodeTiled is not available");
    const size_t es = h->esize();
    h->maps.resize((size_t)2 * h->nruns * 4);
    const CUtensorMapDataType dt =
        h->prec == ACM_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    for (int run = 0; run < h->nruns; ++run) {
        // one map per (buffer, run, field): the run's padded planes, ghost
        // planes included; base = pool + run offset (a multiple of 32
        // elements, so 16-byte aligned)
        const RunDesc &R = h->runs[run];
        cuuint64_t dims[3] = {(cuuint64_t)R.px, (cuuint64_t)R.py, (cuuint64_t)(R.nz + 2 * R.zg)};
        cuuint64_t strides[2] = {(cuuint64_t)(R.px * es), (cuuint64_t)(R.px * R.py * es)};
        cuuint32_t box[3] = {(cuuint32_t)(T3X + 4), (cuuint32_t)(h->tune.t3y + 4), 1};
        cuuint32_t estr[3] = {1, 1, 1};
        for (int b = 0; b < 2; ++b)
            for (int f = 0; f < 4; ++f) {
                void *base = static_cast<char *>(h->buf[b][f]) + (size_t)R.off * es;
                CUresult r = fn(&h->maps[((size_t)b * h->nruns + run) * 4 + f], dt, 3, base, dims,
                                strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS)
                    return fail(h, ACM_ECUDA,
                                "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
            }
    }
    h->maps_ok = true;
    return ACM_OK;
}

void drop_graph(acm_handle *h)
{
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
}

void release(acm_handle *h)
{
    drop_graph(h);
    if (h->own_fields)
        for (int b = 0; b < 2; ++b)
            for (int f = 0; f < NFIELD; ++f)
                if (h->buf[b][f]) cudaFree(h->buf[b][f]);
    if (h->druns) cudaFree(h->druns);
    if (h->dwork) cudaFree(h->dwork);
    if (h->dline) cudaFree(h->dline);
    if (h->derr) cudaFree(h->derr);
    if (h->dpartials) cudaFree(h->dpartials);
    if (h->dout) cudaFree(h->dout);
    if (h->dstage) cudaFree(h->dstage);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    for (void *p : h->scratch)
        if (p) cudaFree(p);
    // a creation that failed part-way leaves null entries
    for (cudaStream_t st : h->side)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
}

bool field_used(const acm_handle *h, int f)
{
    if (f == F_W) return h->dim == 3;
    if (f == F_PHI) return h->two_phase != 0;
    return true;
}

// elements per field pool of a run described by d (each run starts on a
// 32-element, i.e. 128/256-byte, boundary)
size_t run_elems(const RunDesc &d)
{
    const size_t n = (size_t)d.px * d.py * (d.nz + 2 * d.zg);
    return (n + 31) / 32 * 32;
}

// ext != nullptr: acm_create_ext (10 caller-owned buffers, caller's stream)
acm_status create_common(const acm_params *params, int nruns, acm_handle **out,
                         void *const *ext = nullptr, cudaStream_t ext_stream = nullptr)
{
    if (out) *out = nullptr;
    if (!params || !out || nruns < 1) return fail(nullptr, ACM_EINVAL, "null argument or nruns < 1");
    std::string why;
    for (int r = 0; r < nruns; ++r)
        if (validate(params[r], why) != ACM_OK)
            return fail(nullptr, ACM_EINVAL, "run " + std::to_string(r) + ": " + why);
    const acm_params &p0 = params[0];
    if (p0.dim == 3 && (nruns > 1 || p0.bc[4] == ACM_BC_HALO)) {
        // the runs are z-slabs of one grid
        for (int r = 0; r < nruns; ++r) {
            const acm_params &p = params[r];
            if (p.dim != 3 || p.bc[4] != ACM_BC_HALO)
                return fail(nullptr, ACM_EINVAL,
                            "3D batches are sub-domains: every run needs ACM_BC_HALO z faces");
            if (p.nx != p0.nx || p.ny != p0.ny || p.precision != p0.precision ||
                p.dt != p0.dt || p.nu != p0.nu || p.rho0 != p0.rho0 ||
                p.sat_mask != p0.sat_mask || p.g[0] != p0.g[0] || p.g[1] != p0.g[1] ||
                p.g[2] != p0.g[2])
                return fail(nullptr, ACM_EINVAL,
                            "sub-domains must share nx, ny, precision and the physical parameters");
        }
    } else if (nruns > 1) {
        for (int r = 1; r < nruns; ++r) {
            const acm_params &p = params[r];
            if (p.dim != p0.dim || p.precision != p0.precision || p.two_phase != p0.two_phase ||
                p.scheme != p0.scheme)
                return fail(nullptr, ACM_EINVAL,
                            "batch runs must share dim, precision, two_phase, scheme");
        }
    }
    acm_handle *h = new (std::nothrow) acm_handle();
    if (!h) return fail(nullptr, ACM_ENOMEM, "host allocation failed");
    h->nruns = nruns;
    h->dim = p0.dim;
    h->prec = p0.precision;
    h->two_phase = p0.two_phase;
    h->scheme = p0.scheme;
    h->params.assign(params, params + nruns);
    h->have_fields.assign(nruns, 0);
    auto bail = [&](acm_status st) {
        std::string m = h->err;
        release(h);
        delete h;
        return fail(nullptr, st, m);
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        cuda_fail(h, e, "cudaGetDevice");
        return bail(ACM_ECUDA);
    }
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (h->sms <= 0) h->sms = 1;

    // per-run descriptors, pool offsets (each run starts on a 256-byte boundary)
    size_t off = 0;
    long long maxn = 0;
    std::vector<int4> work;
    for (int r = 0; r < nruns; ++r) {
        RunDesc d = describe(params[r]);
        d.off = (long long)off;
        off += run_elems(d);
        if (d.zg) h->halo = true;
        h->runs.push_back(d);
        const long long np = (long long)d.nx * d.ny * d.nz;
        h->npoints.push_back(np);
        maxn = std::max(maxn, np);
        for (int f = 0; f < 4; ++f)
            if (d.bc[f] != ACM_BC_PERIODIC) h->any_wall = 1;
        if (h->dim == 2) {
            const int tx = (d.nx + T2X - 1) / T2X, ty = (d.ny + T2Y - 1) / T2Y;
            for (int j = 0; j < ty; ++j)
                for (int i = 0; i < tx; ++i) {
                    const int x0 = std::min(i * T2X, std::max(d.nx - T2X, 0));
                    const int y0 = std::min(j * T2Y, std::max(d.ny - T2Y, 0));
                    work.push_back(make_int4(r, x0, y0, 0));
                }
        }
    }
    h->pool = off;
    h->nwork = (int)work.size();
    // the line-marching kernel covers single-phase 2D runs that are periodic
    // on all four faces, with a width that is a multiple of its strip
    std::vector<int4> line;
    if (h->dim == 2 && h->two_phase) {
        // two-phase line-marching kernel: periodic runs, strips of
        // line2d_tp_stride() written columns starting at x0 = k stride - 4
        bool ok = true;
        for (const RunDesc &d : h->runs) {
            for (int f = 0; f < 4; ++f) ok &= d.bc[f] == ACM_BC_PERIODIC;
            ok &= d.nx >= 64 && d.ny >= 16;
            h->line_gen |= d.rho0 != 1.0 || d.g[0] != 0.0 || d.g[1] != 0.0;
        }
        const int sw = line2d_tp_stride();
        int rows = line2d_tp_rows();
        auto count = [&](int rr) {
            long long n = 0;
            for (const RunDesc &d : h->runs)
                n += (long long)((d.nx + sw - 1) / sw) * ((d.ny + rr - 1) / rr);
            return n;
        };
        while (ok && rows > 16 && count(rows) < 32LL * h->sms) rows /= 2;
        for (int r = 0; ok && r < nruns; ++r) {
            const RunDesc &d = h->runs[r];
            for (int y0 = 0; y0 < d.ny; y0 += rows)
                for (int x0 = 0; x0 < d.nx; x0 += sw)
                    line.push_back(make_int4(r, x0 - 4, y0, std::min(rows, d.ny - y0)));
        }
    }
    if (h->dim == 2 && !h->two_phase) {
        bool ok = true;
        for (const RunDesc &d : h->runs) {
            for (int f = 0; f < 4; ++f) ok &= d.bc[f] == ACM_BC_PERIODIC;
            ok &= d.nx % line2d_width() == 0 && d.ny >= 4;
            h->line_gen |= d.rho0 != 1.0 || d.g[0] != 0.0 || d.g[1] != 0.0;
        }
        // rows per item: the most (up to line2d_rows()) that still give 32
        // items per SM (two per warp slot at 16 resident warps); short items
        // (down to 4 rows) spread small grids over the GPU
        int rows = line2d_rows();
        auto count = [&](int rr) {
            long long n = 0;
            for (const RunDesc &d : h->runs)
                n += (long long)(d.nx / line2d_width()) * ((d.ny + rr - 1) / rr);
            return n;
        };
        while (ok && rows > 4 && count(rows) < 32LL * h->sms) rows /= 2;
        for (int r = 0; ok && r < nruns; ++r) {
            const RunDesc &d = h->runs[r];
            for (int y0 = 0; y0 < d.ny; y0 += rows)
                for (int x0 = 0; x0 < d.nx; x0 += line2d_width())
                    line.push_back(make_int4(r, x0, y0, std::min(rows, d.ny - y0)));
        }
    }
    h->nline = (int)line.size();
    // the line-marching kernel is the default for FP32 storage; in FP64 its
    // register queue limits it to one CTA per SM and the tile kernel is
    // faster on the grids measured
    h->tune.line2d = h->prec == ACM_FP64 ? 0 : 1;

#define CKB(call)                                    \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) {                     \
            acm_status st_ = cuda_fail(h, e_, #call); \
            return bail(st_);                        \
        }                                            \
    } while (0)

    if (ext) {
        h->stream = ext_stream;
        h->own_stream = false;
    } else {
        CKB(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    if (h->halo && nruns > 1) {
        h->side.assign(nruns - 1, nullptr);
        h->ev.assign(nruns, nullptr);
        for (auto &st : h->side) CKB(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        for (auto &e : h->ev) CKB(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (ext) {
        // caller-owned storage: checked by acm_create_ext, zero-filled here
        h->own_fields = false;
        for (int b = 0; b < 2; ++b)
            for (int f = 0; f < NFIELD; ++f)
                if (field_used(h, f)) {
                    h->buf[b][f] = ext[NFIELD * b + f];
                    CKB(cudaMemsetAsync(h->buf[b][f], 0, h->pool * h->esize(), h->stream));
                }
        CKB(cudaStreamSynchronize(h->stream));
    } else {
        for (int b = 0; b < 2; ++b)
            for (int f = 0; f < NFIELD; ++f)
                if (field_used(h, f)) {
                    CKB(cudaMalloc(&h->buf[b][f], h->pool * h->esize()));
                    CKB(cudaMemset(h->buf[b][f], 0, h->pool * h->esize()));
                }
    }
    if (h->dim == 3 && h->two_phase)
        for (void *&p : h->scratch) {
            CKB(cudaMalloc(&p, h->pool * h->esize()));
            CKB(cudaMemset(p, 0, h->pool * h->esize()));
        }
    CKB(cudaMalloc(&h->druns, sizeof(RunDesc) * nruns));
    CKB(cudaMemcpy(h->druns, h->runs.data(), sizeof(RunDesc) * nruns, cudaMemcpyHostToDevice));
    if (!work.empty()) {
        CKB(cudaMalloc(&h->dwork, sizeof(int4) * work.size()));
        CKB(cudaMemcpy(h->dwork, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice));
    }
    if (!line.empty()) {
        CKB(cudaMalloc(&h->dline, sizeof(int4) * line.size()));
        CKB(cudaMemcpy(h->dline, line.data(), sizeof(int4) * line.size(), cudaMemcpyHostToDevice));
    }
    CKB(cudaMalloc(&h->derr, sizeof(unsigned)));
    CKB(cudaMemset(h->derr, 0, sizeof(unsigned)));
    const long long per_run_blocks = (maxn + 255) / 256;
    h->red_blocks = (int)std::max<long long>(
        1, std::min<long long>(per_run_blocks, nruns == 1 ? 4LL * h->sms : 16LL));
    // room for the partials of every reduction: 8 (acm_reduce_mass), 2 per
    // block (acm_reduce_error) or LAPLACE_PARTIALS (acm_reduce_laplace)
    CKB(cudaMalloc(&h->dpartials,
                   sizeof(double) * LAPLACE_PARTIALS * (size_t)h->red_blocks * nruns));
    CKB(cudaMalloc(&h->dout, sizeof(double) * 8 * nruns));
    CKB(cudaMalloc(&h->dstage, sizeof(double) * (size_t)maxn));
    if (build_maps(h) != ACM_OK) return bail(ACM_ECUDA);
    // resolve launch attributes now, not inside a later stream capture
    if (h->dim == 2) {
        if (h->prec == ACM_FP64) step2d_max_blocks_per_sm<double>(h->two_phase);
        else step2d_max_blocks_per_sm<float>(h->two_phase);
        if (h->nline > 0 && !h->two_phase) {
            if (h->prec == ACM_FP64) line2d_prepare<double>();
            else line2d_prepare<float>();
        }
        if (h->nline > 0 && h->two_phase) {
            if (h->prec == ACM_FP64) line2d_tp_prepare<double>();
            else line2d_tp_prepare<float>();
        }
        if (h->scheme == ACM_SCHEME_MAMES) {
            if (h->prec == ACM_FP64) mames2d_max_blocks_per_sm<double>();
            else mames2d_max_blocks_per_sm<float>();
        }
    } else if (h->two_phase) {
        if (h->prec == ACM_FP64) tp3d_prepare<double>();
        else tp3d_prepare<float>();
    } else {
        for (int t3y : {8, 16}) {
            if (h->prec == ACM_FP64) step3d_max_blocks_per_sm<double>(t3y);
            else step3d_max_blocks_per_sm<float>(t3y);
        }
    }
    *out = h;
    return ACM_OK;
}

template <typename T>
Fields<T> fields_of(acm_handle *h, int b)
{
    Fields<T> f;
    for (int k = 0; k < NFIELD; ++k) f.f[k] = static_cast<T *>(h->buf[b][k]);
    return f;
}

template <typename T>
cudaError_t one_step(acm_handle *h, int from)
{
    Fields<T> in = fields_of<T>(h, from), out = fields_of<T>(h, 1 - from);
    if (h->dim == 3 && h->two_phase)
        return launch_tp3d<T>(h->runs[0], in, out, static_cast<T *>(h->scratch[0]),
                              static_cast<T *>(h->scratch[1]), static_cast<T *>(h->scratch[2]),
                              h->derr, h->sms, h->stream);
    if (h->dim == 3) {
        cudaError_t e = cudaSuccess;
        if (h->halo) {
            const RunDesc &R = h->runs[0];
            e = launch_halo<T>(h->druns, h->nruns, R.px * R.py, in, h->stream);
        }
        // one launch per sub-domain (a single launch for one periodic grid);
        // the slabs write disjoint planes, so their launches run concurrently
        // on forked streams and the next step waits for all of them
        const bool fork = !h->side.empty();
        if (fork && e == cudaSuccess) e = cudaEventRecord(h->ev[0], h->stream);
        for (int r = 0; r < h->nruns && e == cudaSuccess; ++r) {
            cudaStream_t st = r == 0 ? h->stream : h->side[r - 1];
            if (r > 0) e = cudaStreamWaitEvent(st, h->ev[0], 0);
            if (e == cudaSuccess)
                e = launch_step3d<T>(&h->maps[((size_t)from * h->nruns + r) * 4], out,
                                     h->runs[r], h->derr, h->tune.zchunks, h->tune.t3y, h->sms,
                                     st);
            if (r > 0 && e == cudaSuccess) e = cudaEventRecord(h->ev[r], st);
        }
        for (int r = 1; r < h->nruns && fork && e == cudaSuccess; ++r)
            e = cudaStreamWaitEvent(h->stream, h->ev[r], 0);
        return e;
    }
    int blocks = h->tune.blocks;
    if (h->scheme == ACM_SCHEME_MAMES) {
        if (blocks <= 0) blocks = h->sms * mames2d_max_blocks_per_sm<T>();
        return launch_mames2d<T>(h->druns, h->dwork, h->nwork, in, out, h->derr, blocks,
                                 h->stream);
    }
    if (h->nline > 0 && h->tune.line2d)
        return h->two_phase ? launch_line2d_tp<T>(h->druns, h->dline, h->nline, h->line_gen, in,
                                                  out, h->derr, h->stream)
                            : launch_line2d<T>(h->druns, h->dline, h->nline, h->line_gen, in,
                                               out, h->derr, h->stream);
    if (blocks <= 0) blocks = h->sms * step2d_max_blocks_per_sm<T>(h->two_phase);
    return launch_step2d<T>(h->druns, h->dwork, h->nwork, h->two_phase, in, out, h->derr, blocks,
                            h->stream);
}

cudaError_t step_once(acm_handle *h, int from)
{
    return h->prec == ACM_FP64 ? one_step<double>(h, from) : one_step<float>(h, from);
}

acm_status ensure_graph(acm_handle *h)
{
    if (h->gexec) return ACM_OK;
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < h->tune.graph_steps && le == cudaSuccess; ++k) le = step_once(h, k & 1);
    cudaError_t ee = cudaStreamEndCapture(h->stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, le, "kernel launch during capture");
    }
    if (ee != cudaSuccess) return cuda_fail(h, ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        h->gexec = nullptr;
        return cuda_fail(h, ie, "cudaGraphInstantiate");
    }
    return ACM_OK;
}

acm_status check_flags(acm_handle *h)
{
    // every step kernel ORs ERR_NONFINITE into the error word itself
    unsigned flags = 0;
    CK(h, cudaMemcpyAsync(&flags, h->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->sticky |= flags;
    if (h->sticky & ERR_TIMEOUT) return fail(h, ACM_ETIMEOUT, "a device-side wait timed out");
    if (h->sticky & ERR_NONFINITE)
        return fail(h, ACM_EUNSTABLE, "non-finite values in the fields (numerical blow-up)");
    return ACM_OK;
}

}  // namespace

namespace {

// box-filter restriction of fine fields onto a coarse grid (2D, one run per
// blockIdx.y): coarse = mean of the factor x factor fine nodes it covers
template <typename TF, typename TC>
__global__ void k_restrict(const RunDesc *__restrict__ fr, Fields<TF> fine, const RunDesc *cr,
                           Fields<TC> coarse, int factor, double us, double rs, float *out,
                           float sr, float su, int nxc, int nyc)
{
    const int run = blockIdx.y;
    const RunDesc &F = fr[run];
    const long long nc = (long long)nxc * nyc;
    const double inv = 1.0 / ((double)factor * factor);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nc;
         i += (long long)gridDim.x * blockDim.x) {
        const int yc = (int)(i / nxc), xc = (int)(i - (long long)yc * nxc);
        double sr_ = 0.0, su_ = 0.0, sv_ = 0.0;
        for (int a = 0; a < factor; ++a)
            for (int b = 0; b < factor; ++b) {
                const long long k = F.off + (long long)(yc * factor + a) * F.nx + xc * factor + b;
                sr_ += (double)fine.f[F_R][k];
                su_ += (double)fine.f[F_U][k];
                sv_ += (double)fine.f[F_V][k];
            }
        // unit change to the coarse lattice: velocity times us, density
        // deviation (the pressure signal) times rs
        const double r = sr_ * inv * rs, u = su_ * inv * us, v = sv_ * inv * us;
        if (cr) {
            const RunDesc &C = cr[run];
            const long long k = C.off + i;
            coarse.f[F_R][k] = (TC)r;
            coarse.f[F_U][k] = (TC)u;
            coarse.f[F_V][k] = (TC)v;
        }
        if (out) {
            float *o = out + (long long)run * 3 * nc;
            o[i] = (float)(r * sr);
            o[nc + i] = (float)(u * su);
            o[2 * nc + i] = (float)(v * su);
        }
    }
}

template <typename TF, typename TC>
cudaError_t restrict_launch(acm_handle *f, acm_handle *c, int factor, double us, double rs,
                            float *out, float sr, float su, int nxc, int nyc)
{
    Fields<TF> ff;
    Fields<TC> cf;
    for (int k = 0; k < NFIELD; ++k) {
        ff.f[k] = static_cast<TF *>(f->buf[f->cur][k]);
        cf.f[k] = c ? static_cast<TC *>(c->buf[c->cur][k]) : nullptr;
    }
    dim3 grid(256, f->nruns);
    k_restrict<TF, TC><<<grid, 256, 0, f->stream>>>(f->druns, ff, c ? c->druns : nullptr, cf,
                                                    factor, us, rs, out, sr, su, nxc, nyc);
    return cudaGetLastError();
}

}  // namespace

namespace acm {
cudaError_t order_streams(cudaStream_t prev, cudaStream_t next)
{
    if (prev == next) return cudaSuccess;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev, prev);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(next, ev, 0);
    cudaEventDestroy(ev);  // released once the wait has been satisfied
    return e;
}

acm_status handle_fields_f32(acm_handle *h, int run, float **r, float **u, float **v, int *nx,
                             int *ny)
{
    if (!h || run < 0 || run >= h->nruns || h->dim != 2 || h->prec != ACM_FP32_DEV)
        return ACM_EINVAL;
    const RunDesc &R = h->runs[run];
    *r = static_cast<float *>(h->buf[h->cur][F_R]) + R.off;
    *u = static_cast<float *>(h->buf[h->cur][F_U]) + R.off;
    *v = static_cast<float *>(h->buf[h->cur][F_V]) + R.off;
    *nx = R.nx;
    *ny = R.ny;
    return ACM_OK;
}
}  // namespace acm

extern "C" {

acm_status acm_create(const acm_params *params, acm_handle **out)
{
    return create_common(params, 1, out);
}

acm_status acm_batch_create(const acm_params *params, int nruns, acm_handle **out)
{
    return create_common(params, nruns, out);
}

acm_status acm_storage_elems(const acm_params *params, size_t *elems)
{
    if (!params || !elems) return fail(nullptr, ACM_EINVAL, "null argument");
    std::string why;
    if (validate(*params, why) != ACM_OK) return fail(nullptr, ACM_EINVAL, why);
    *elems = run_elems(describe(*params));
    return ACM_OK;
}

acm_status acm_create_ext(const acm_params *params, void *const *dev_fields, void *stream,
                          acm_handle **out)
{
    if (out) *out = nullptr;
    if (!params || !dev_fields || !out) return fail(nullptr, ACM_EINVAL, "null argument");
    std::string why;
    if (validate(*params, why) != ACM_OK) return fail(nullptr, ACM_EINVAL, why);
    const bool used[NFIELD] = {true, true, true, params->dim == 3, params->two_phase != 0};
    for (int b = 0; b < 2; ++b)
        for (int f = 0; f < NFIELD; ++f) {
            const void *p = dev_fields[NFIELD * b + f];
            if (used[f] && !p)
                return fail(nullptr, ACM_EINVAL, "missing device buffer for a field the run has");
            if (!used[f] && p)
                return fail(nullptr, ACM_EINVAL,
                            "device buffer given for a field the run does not have");
            if (p && (reinterpret_cast<uintptr_t>(p) & 255))
                return fail(nullptr, ACM_EINVAL, "device buffers must start on 256-byte boundaries");
        }
    return create_common(params, 1, out, dev_fields, static_cast<cudaStream_t>(stream));
}

int acm_current_buffer(const acm_handle *h) { return h ? h->cur : -1; }

acm_status acm_stability_ratio(const acm_params *params, const double *u, const double *v,
                               const double *w, size_t n, double *ratio)
{
    if (!params || !u || !v || !ratio || (params->dim == 3 && !w))
        return fail(nullptr, ACM_EINVAL, "null argument");
    if (!(params->dt > 0) || !(params->nu >= 0) || (params->dim != 2 && params->dim != 3))
        return fail(nullptr, ACM_EINVAL, "bad dim, dt or nu");
    double q = 0.0;
    for (size_t i = 0; i < n; ++i) {
        double s = u[i] * u[i] + v[i] * v[i];
        if (params->dim == 3) s += w[i] * w[i];
        if (!(s <= q)) q = s;  // NaN propagates
    }
    const double nu = params->nu, dt = params->dt;
    const double adv = nu > 0 ? q * dt / (2.0 * nu) : (q > 0 || std::isnan(q) ? INFINITY : 0.0);
    const double dif = 2.0 * params->dim * nu * dt;
    *ratio = std::isnan(adv) ? adv : std::max(adv, dif);
    return ACM_OK;
}

acm_status acm_set_stream(acm_handle *h, void *stream)
{
    if (!h) return fail(nullptr, ACM_EINVAL, "null handle");
    const cudaStream_t next = static_cast<cudaStream_t>(stream);
    CK(h, cudaSetDevice(h->device));
    drop_graph(h);
    if (h->own_stream && h->stream) {
        cudaStreamSynchronize(h->stream);
        cudaStreamDestroy(h->stream);
    } else {
        // a caller's stream: the work already queued on it comes first
        CK(h, order_streams(h->stream, next));
    }
    h->own_stream = false;
    h->stream = next;
    return ACM_OK;
}

int acm_nruns(const acm_handle *h) { return h ? h->nruns : 0; }

int64_t acm_step_count(const acm_handle *h) { return h ? h->steps : -1; }

acm_status acm_set_tuning(acm_handle *h, int key, int value)
{
    if (!h) return fail(nullptr, ACM_EINVAL, "null handle");
    switch (key) {
    case ACM_TUNE_ZCHUNKS:
        if (value < 0) return fail(h, ACM_EINVAL, "zchunks must be >= 0");
        h->tune.zchunks = value;
        break;
    case ACM_TUNE_T3Y:
        if (value != 8 && value != 16) return fail(h, ACM_EINVAL, "t3y must be 8 or 16");
        if (value != h->tune.t3y) {
            cudaSetDevice(h->device);
            CK(h, cudaStreamSynchronize(h->stream));
            h->tune.t3y = value;
            if (build_maps(h) != ACM_OK) return ACM_ECUDA;
        }
        break;
    case ACM_TUNE_GRAPH_STEPS:
        if (value < 0 || (value & 1)) return fail(h, ACM_EINVAL, "graph_steps must be even >= 0");
        h->tune.graph_steps = value;
        break;
    case ACM_TUNE_BLOCKS:
        if (value < 0) return fail(h, ACM_EINVAL, "blocks must be >= 0");
        h->tune.blocks = value;
        break;
    case ACM_TUNE_LINE2D:
        if (value != 0 && value != 1) return fail(h, ACM_EINVAL, "line2d must be 0 or 1");
        h->tune.line2d = value;
        break;
    default:
        return fail(h, ACM_EINVAL, "unknown tuning key");
    }
    drop_graph(h);
    return ACM_OK;
}

int acm_get_tuning(const acm_handle *h, int key)
{
    if (!h) return -1;
    switch (key) {
    case ACM_TUNE_ZCHUNKS: return h->tune.zchunks;
    case ACM_TUNE_T3Y: return h->tune.t3y;
    case ACM_TUNE_GRAPH_STEPS: return h->tune.graph_steps;
    case ACM_TUNE_BLOCKS: return h->tune.blocks;
    case ACM_TUNE_LINE2D: return h->tune.line2d;
    default: return -1;
    }
}

acm_status acm_autotune(acm_handle *h, int nsteps, double *best_ms_per_step)
{
    NvtxRange nvtx_("acm_autotune");
    if (!h) return fail(nullptr, ACM_EINVAL, "null handle");
    if (nsteps < 1) return fail(h, ACM_EINVAL, "nsteps must be >= 1");
    for (int r = 0; r < h->nruns; ++r)
        if (!h->have_fields[r]) return fail(h, ACM_ESTATE, "acm_set_fields not called for every run");
    if (h->sticky) return fail(h, ACM_EUNSTABLE, "fields already non-finite");
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));

    // candidate launch shapes
    struct Cand { int t3y, zchunks, blocks, line2d; };
    std::vector<Cand> cands;
    if (h->dim == 3) {
        const int nz = h->runs[0].nz;
        const int zc_opts[4] = {0, std::max(1, nz / 8), std::max(1, nz / 32), std::max(1, nz / 64)};
        for (int t3y : {16, 8})
            for (int zc : zc_opts) {
                bool dup = false;
                for (const Cand &c : cands) dup |= (c.t3y == t3y && c.zchunks == zc);
                if (!dup) cands.push_back({t3y, zc, 0, 0});
            }
    } else {
        const bool mames = h->scheme == ACM_SCHEME_MAMES;
        const int per_sm =
            h->prec == ACM_FP64
                ? (mames ? mames2d_max_blocks_per_sm<double>()
                         : step2d_max_blocks_per_sm<double>(h->two_phase))
                : (mames ? mames2d_max_blocks_per_sm<float>()
                         : step2d_max_blocks_per_sm<float>(h->two_phase));
        for (int k = 1; k <= per_sm; ++k) cands.push_back({h->tune.t3y, 0, k * h->sms, 0});
        if (h->nline > 0 && !mames) cands.push_back({h->tune.t3y, 0, 0, 1});
    }

    // keep the state: trial steps run on a copy
    const size_t bytes = h->pool * h->esize();
    void *save[NFIELD] = {};
    acm_status st = ACM_OK;
    for (int f = 0; f < NFIELD && st == ACM_OK; ++f) {
        if (!field_used(h, f)) continue;
        cudaError_t e = cudaMalloc(&save[f], bytes);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(save[f], h->buf[h->cur][f], bytes, cudaMemcpyDeviceToDevice,
                                h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "autotune state copy");
    }
    const int cur0 = h->cur;
    const Tuning keep = h->tune;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 1e300;
    Cand bestc = {keep.t3y, keep.zchunks, keep.blocks, keep.line2d};
    if (st == ACM_OK) {
        cudaError_t ee = cudaEventCreate(&e0);
        if (ee == cudaSuccess) ee = cudaEventCreate(&e1);
        if (ee != cudaSuccess) st = cuda_fail(h, ee, "cudaEventCreate");
    }
    for (size_t i = 0; i < cands.size() && st == ACM_OK; ++i) {
        const Cand &c = cands[i];
        if (h->dim == 3 && c.t3y != h->tune.t3y) {
            h->tune.t3y = c.t3y;
            if (build_maps(h) != ACM_OK) {
                st = ACM_ECUDA;
                break;
            }
        }
        h->tune.zchunks = c.zchunks;
        h->tune.blocks = c.blocks;
        h->tune.line2d = c.line2d;
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {  // warm-up
            e = step_once(h, h->cur);
            h->cur ^= 1;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
            e = step_once(h, h->cur);
            h->cur ^= 1;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            st = cuda_fail(h, e, "autotune trial");
            break;
        }
        if (ms / nsteps < best) {
            best = ms / nsteps;
            bestc = c;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // restore the state and apply the winner
    h->cur = cur0;
    for (int f = 0; f < NFIELD; ++f) {
        if (!save[f]) continue;
        if (st == ACM_OK) {
            cudaError_t e = cudaMemcpyAsync(h->buf[cur0][f], save[f], bytes,
                                            cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) st = cuda_fail(h, e, "autotune restore");
        }
    }
    cudaStreamSynchronize(h->stream);
    for (int f = 0; f < NFIELD; ++f)
        if (save[f]) cudaFree(save[f]);
    h->tune = keep;
    if (st == ACM_OK) {
        h->tune.zchunks = bestc.zchunks;
        h->tune.blocks = bestc.blocks;
        h->tune.line2d = bestc.line2d;
        if (h->dim == 3) h->tune.t3y = bestc.t3y;
    }
    if (h->dim == 3 && build_maps(h) != ACM_OK && st == ACM_OK) st = ACM_ECUDA;
    drop_graph(h);
    cudaMemsetAsync(h->derr, 0, sizeof(unsigned), h->stream);
    cudaStreamSynchronize(h->stream);
    if (best_ms_per_step) *best_ms_per_step = st == ACM_OK ? best : 0.0;
    return st;
}

acm_status acm_set_fields(acm_handle *h, int run, const double *rho, const double *u,
                          const double *v, const double *w, const double *phi)
{
    NvtxRange nvtx_("acm_set_fields");
    if (!h) return fail(nullptr, ACM_EINVAL, "null handle");
    if (run < 0 || run >= h->nruns) return fail(h, ACM_EINVAL, "run index out of range");
    if (!rho || !u || !v || (h->dim == 3 && !w) || (h->two_phase && !phi))
        return fail(h, ACM_EINVAL, "missing field");
    CK(h, cudaSetDevice(h->device));
    const RunDesc &R = h->runs[run];
    const size_t n = (size_t)h->npoints[run];
    const double *src[NFIELD] = {rho, u, v, w, phi};
    for (int f = 0; f < NFIELD; ++f) {
        if (!field_used(h, f)) continue;
        const double shift = f == F_R ? R.rho0 : 0.0;
        CK(h, cudaMemcpyAsync(h->dstage, src[f], n * sizeof(double), cudaMemcpyHostToDevice,
                              h->stream));
        cudaError_t e = h->prec == ACM_FP64
                            ? launch_import<double>(h->dstage,
                                                    static_cast<double *>(h->buf[h->cur][f]), R,
                                                    h->dim, shift, h->stream)
                            : launch_import<float>(h->dstage, static_cast<float *>(h->buf[h->cur][f]),
                                                   R, h->dim, shift, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "import kernel");
    }
    CK(h, cudaMemsetAsync(h->derr, 0, sizeof(unsigned), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->sticky = 0;
    h->steps = 0;
    h->have_fields[run] = 1;
    // stability pre-check of the initial velocity: a warning, not an error
    double ratio = 0.0;
    h->err.clear();
    if (acm_stability_ratio(&h->params[run], u, v, w, n, &ratio) == ACM_OK && !(ratio <= 1.0)) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "warning: run %d is expected to be unstable: max(|u|^2 dt / (2 nu), "
                      "2 dim nu dt) = %.3g > 1 on the initial field",
                      run, ratio);
        h->err = msg;
    }
    return ACM_OK;
}

acm_status acm_step(acm_handle *h, int64_t nsteps)
{
    NvtxRange nvtx_("acm_step");
    if (!h) return fail(nullptr, ACM_EINVAL, "null handle");
    if (nsteps < 0) return fail(h, ACM_EINVAL, "nsteps must be >= 0");
    for (int r = 0; r < h->nruns; ++r)
        if (!h->have_fields[r]) return fail(h, ACM_ESTATE, "acm_set_fields not called for every run");
    if (h->sticky & ERR_TIMEOUT) return fail(h, ACM_ETIMEOUT, "a device-side wait timed out");
    if (h->sticky & ERR_NONFINITE) return fail(h, ACM_EUNSTABLE, "fields already non-finite");
    CK(h, cudaSetDevice(h->device));
    int64_t left = nsteps;
    const int G = h->tune.graph_steps;
    if (h->cur == 1 && left > 0) {
        CK(h, step_once(h, 1));
        h->cur = 0;
        --left;
    }
    if (G > 0 && h->stream != nullptr && left >= G) {
        acm_status st = ensure_graph(h);
        if (st != ACM_OK) return st;
        while (left >= G) {
            CK(h, cudaGraphLaunch(h->gexec, h->stream));
            left -= G;
        }
    }
    while (left > 0) {
        CK(h, step_once(h, h->cur));
        h->cur ^= 1;
        --left;
    }
    h->steps += nsteps;
    return ACM_OK;
}

acm_status acm_sync(acm_handle *h)
{
    NvtxRange nvtx_("acm_sync");
    if (!h) return fail(nullptr, ACM_EINVAL, "null handle");
    CK(h, cudaSetDevice(h->device));
    return check_flags(h);
}

acm_status acm_fields(acm_handle *h, int run, double *rho, double *u, double *v, double *w,
                      double *phi)
{
    NvtxRange nvtx_("acm_fields");
    if (!h) return fail(nullptr, ACM_EINVAL, "null handle");
    if (run < 0 || run >= h->nruns) return fail(h, ACM_EINVAL, "run index out of range");
    CK(h, cudaSetDevice(h->device));
    const RunDesc &R = h->runs[run];
    const size_t n = (size_t)h->npoints[run];
    double *dst[NFIELD] = {rho, u, v, w, phi};
    for (int f = 0; f < NFIELD; ++f) {
        if (!dst[f] || !field_used(h, f)) continue;
        const double shift = f == F_R ? R.rho0 : 0.0;
        cudaError_t e =
            h->prec == ACM_FP64
                ? launch_export<double>(static_cast<const double *>(h->buf[h->cur][f]), h->dstage,
                                        R, h->dim, shift, h->stream)
                : launch_export<float>(static_cast<const float *>(h->buf[h->cur][f]), h->dstage, R,
                                       h->dim, shift, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "export kernel");
        CK(h, cudaMemcpyAsync(dst[f], h->dstage, n * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
    }
    return check_flags(h);
}

acm_status acm_reduce_mass(acm_handle *h, double *out)
{
    NvtxRange nvtx_("acm_reduce_mass");
    if (!h || !out) return fail(h, ACM_EINVAL, "null argument");
    CK(h, cudaSetDevice(h->device));
    const int prev = 1 - h->cur;
    const bool have_prev = h->steps > 0;
    cudaError_t e;
    if (h->prec == ACM_FP64) {
        const double *pu = have_prev ? static_cast<const double *>(h->buf[prev][F_U]) : nullptr;
        const double *pv = have_prev ? static_cast<const double *>(h->buf[prev][F_V]) : nullptr;
        const double *pw = have_prev ? static_cast<const double *>(h->buf[prev][F_W]) : nullptr;
        e = launch_reduce<double>(h->druns, h->nruns, h->dim, fields_of<double>(h, h->cur), pu, pv,
                                  pw, h->dpartials, h->red_blocks, h->dout, h->stream);
    } else {
        const float *pu = have_prev ? static_cast<const float *>(h->buf[prev][F_U]) : nullptr;
        const float *pv = have_prev ? static_cast<const float *>(h->buf[prev][F_V]) : nullptr;
        const float *pw = have_prev ? static_cast<const float *>(h->buf[prev][F_W]) : nullptr;
        e = launch_reduce<float>(h->druns, h->nruns, h->dim, fields_of<float>(h, h->cur), pu, pv,
                                 pw, h->dpartials, h->red_blocks, h->dout, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "reduction kernels");
    CK(h, cudaMemcpyAsync(out, h->dout, sizeof(double) * 8 * h->nruns, cudaMemcpyDeviceToHost,
                          h->stream));
    return check_flags(h);
}

acm_status acm_reduce_error(acm_handle *h, int run, const double *u_ref, const double *v_ref,
                            const double *w_ref, double *out)
{
    NvtxRange nvtx_("acm_reduce_error");
    if (!h || !out) return fail(h, ACM_EINVAL, "null argument");
    if (run < 0 || run >= h->nruns) return fail(h, ACM_EINVAL, "run index out of range");
    CK(h, cudaSetDevice(h->device));
    const RunDesc &R = h->runs[run];
    const size_t n = (size_t)h->npoints[run];
    const double *refs[3] = {u_ref, v_ref, h->dim == 3 ? w_ref : nullptr};
    double res[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) {
        if (!refs[a]) continue;
        CK(h, cudaMemcpyAsync(h->dstage, refs[a], n * sizeof(double), cudaMemcpyHostToDevice,
                              h->stream));
        cudaError_t e =
            h->prec == ACM_FP64
                ? launch_error_l2<double>(R, static_cast<const double *>(h->buf[h->cur][F_U + a]),
                                          h->dstage, h->dpartials, h->red_blocks, h->dout + a,
                                          h->stream)
                : launch_error_l2<float>(R, static_cast<const float *>(h->buf[h->cur][F_U + a]),
                                         h->dstage, h->dpartials, h->red_blocks, h->dout + a,
                                         h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "error kernels");
        // the staging buffer is reused by the next component
        CK(h, cudaMemcpyAsync(&res[a], h->dout + a, sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    for (int a = 0; a < 3; ++a) out[a] = res[a];
    return check_flags(h);
}

acm_status acm_reduce_laplace(acm_handle *h, double *out)
{
    NvtxRange nvtx_("acm_reduce_laplace");
    if (!h || !out) return fail(h, ACM_EINVAL, "null argument");
    if (!h->two_phase) return fail(h, ACM_EINVAL, "Laplace diagnostics need a two-phase handle");
    CK(h, cudaSetDevice(h->device));
    cudaError_t e =
        h->prec == ACM_FP64
            ? launch_laplace<double>(h->druns, h->nruns, h->dim,
                                     static_cast<const double *>(h->buf[h->cur][F_PHI]),
                                     static_cast<const double *>(h->buf[h->cur][F_R]),
                                     h->dpartials, h->red_blocks, h->dout, h->stream)
            : launch_laplace<float>(h->druns, h->nruns, h->dim,
                                    static_cast<const float *>(h->buf[h->cur][F_PHI]),
                                    static_cast<const float *>(h->buf[h->cur][F_R]),
                                    h->dpartials, h->red_blocks, h->dout, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "Laplace kernels");
    CK(h, cudaMemcpyAsync(out, h->dout, sizeof(double) * 8 * h->nruns, cudaMemcpyDeviceToHost,
                          h->stream));
    return check_flags(h);
}

acm_status acm_restrict(acm_handle *fine, acm_handle *coarse, int factor, double u_scale,
                        double rho_scale, float *out_dev, const float *scales3)
{
    if (!fine || factor < 1 || (!coarse && !out_dev) || (out_dev && !scales3))
        return fail(fine, ACM_EINVAL, "bad restrict arguments");
    if (fine->dim != 2) return fail(fine, ACM_EINVAL, "restriction is 2D only");
    const RunDesc &F0 = fine->runs[0];
    if (F0.nx % factor || F0.ny % factor) return fail(fine, ACM_EINVAL, "factor must divide the grid");
    const int nxc = F0.nx / factor, nyc = F0.ny / factor;
    for (int r = 0; r < fine->nruns; ++r)
        if (fine->runs[r].nx != F0.nx || fine->runs[r].ny != F0.ny)
            return fail(fine, ACM_EINVAL, "fine runs must share one grid size");
    if (coarse) {
        if (coarse->dim != 2 || coarse->nruns != fine->nruns || coarse->two_phase)
            return fail(coarse, ACM_EINVAL, "coarse handle must be 2D single-phase, same runs");
        for (int r = 0; r < coarse->nruns; ++r)
            if (coarse->runs[r].nx != nxc || coarse->runs[r].ny != nyc)
                return fail(coarse, ACM_EINVAL, "coarse grid must be the fine grid / factor");
    }
    CK(fine, cudaSetDevice(fine->device));
    if (coarse) CK(fine, cudaStreamSynchronize(coarse->stream));
    const float sr = out_dev ? scales3[0] : 1.f, su = out_dev ? scales3[1] : 1.f;
    cudaError_t e;
    const bool f64 = fine->prec == ACM_FP64, c64 = coarse ? coarse->prec == ACM_FP64 : false;
    const double us = u_scale, rs = rho_scale;
    if (f64 && c64)
        e = restrict_launch<double, double>(fine, coarse, factor, us, rs, out_dev, sr, su, nxc, nyc);
    else if (f64)
        e = restrict_launch<double, float>(fine, coarse, factor, us, rs, out_dev, sr, su, nxc, nyc);
    else if (c64)
        e = restrict_launch<float, double>(fine, coarse, factor, us, rs, out_dev, sr, su, nxc, nyc);
    else
        e = restrict_launch<float, float>(fine, coarse, factor, us, rs, out_dev, sr, su, nxc, nyc);
    if (e != cudaSuccess) return cuda_fail(fine, e, "restriction kernel");
    CK(fine, cudaStreamSynchronize(fine->stream));
    if (coarse) {
        coarse->steps = 0;
        coarse->sticky = 0;
        for (int r = 0; r < coarse->nruns; ++r) coarse->have_fields[r] = 1;
        CK(coarse, cudaMemset(coarse->derr, 0, sizeof(unsigned)));
    }
    return ACM_OK;
}

acm_status acm_destroy(acm_handle *h)
{
    if (!h) return ACM_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
    return ACM_OK;
}

const char *acm_last_error(const acm_handle *h)
{
    return h ? h->err.c_str() : g_thread_err.c_str();
}

}  // extern "C"
