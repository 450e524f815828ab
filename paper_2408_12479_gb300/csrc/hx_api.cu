// hx_api.cu -- implementation of the C ABI declared in include/hx.h: contexts,
// mesh setup (1D rules, fibre structure tensors, geometry), quadrature-point
// caches, operator dispatch to the per-degree kernel units, the
// Chebyshev-Jacobi smoother, power iteration and the graph-captured FP64 CG.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <cmath>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hx_internal.h"
#include "hx_vec.h"

// per-(degree, precision) kernel units
#define HX_DECL(P)                                   \
    extern const hx::PrecOps *hx_prec_ops_p##P##_f64(); \
    extern const hx::PrecOps *hx_prec_ops_p##P##_f32();
HX_DECL(1)
HX_DECL(2)
HX_DECL(3)
HX_DECL(4)
HX_DECL(5)
HX_DECL(6)
#undef HX_DECL
extern const hx::BatchOps *hx_batch_ops_f64();
extern const hx::BatchOps *hx_batch_ops_f32();

namespace hx {
const BatchOps *batch_ops(int prec) { return prec == HX_FP64 ? hx_batch_ops_f64() : hx_batch_ops_f32(); }
const PrecOps *prec_ops(int p, int prec) {
#define HX_CASE(P) \
    case P:        \
        return prec == HX_FP64 ? hx_prec_ops_p##P##_f64() : hx_prec_ops_p##P##_f32();
    switch (p) {
        HX_CASE(1)
        HX_CASE(2)
        HX_CASE(3)
        HX_CASE(4)
        HX_CASE(5)
        HX_CASE(6)
        default:
            return nullptr;
    }
#undef HX_CASE
}
}  // namespace hx

namespace {

// ---------------------------------------------------------------------------
// 1D rules on [0, 1]
// ---------------------------------------------------------------------------
// Legendre P_n and P_n' on [-1, 1] by the three-term recurrence
void legendre(int n, double x, double &P, double &dP) {
    double p0 = 1.0, p1 = x;
    if (n == 0) {
        P = 1.0;
        dP = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    P = p1;
    dP = n * (x * p1 - p0) / (x * x - 1.0);
}

// Gauss-Legendre: roots of P_n by Newton from Chebyshev-like guesses
void gauss_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double t = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(n, t, P, dP);
            const double dt = P / dP;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        double P, dP;
        legendre(n, t, P, dP);
        x[i] = 0.5 * (t + 1.0);
        w[i] = 1.0 / ((1.0 - t * t) * dP * dP);  // 2/((1-t^2)P'^2), halved for [0,1]
    }
}

// Gauss-Lobatto-Legendre: end points and the roots of P_p', found by Newton on
// P_p' with P_p'' = (2t P_p' - p(p+1) P_p)/(1 - t^2)
std::vector<double> gll_points(int p) {
    std::vector<double> x(p + 1);
    x[0] = 0.0;
    x[p] = 1.0;
    for (int i = 1; i < p; ++i) {
        double t = -std::cos(M_PI * i / p);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(p, t, P, dP);
            const double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
            const double dt = dP / d2P;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        x[i] = 0.5 * (t + 1.0);
    }
    return x;
}

double lagrange(const std::vector<double> &xs, int a, double x) {
    double v = 1.0;
    for (size_t b = 0; b < xs.size(); ++b)
        if ((int)b != a) v *= (x - xs[b]) / (xs[a] - xs[b]);
    return v;
}

double lagrange_d(const std::vector<double> &xs, int a, double x) {
    double s = 0.0;
    for (size_t m = 0; m < xs.size(); ++m) {
        if ((int)m == a) continue;
        double v = 1.0 / (xs[a] - xs[m]);
        for (size_t b = 0; b < xs.size(); ++b)
            if ((int)b != a && b != m) v *= (x - xs[b]) / (xs[a] - xs[b]);
        s += v;
    }
    return s;
}

struct Tables {
    std::vector<double> B, D, Gd, w, geoV, geoD, geoVn;
};

Tables make_tables(int p) {
    const int n = p + 1;
    Tables t;
    std::vector<double> xq, wq;
    gauss_rule(n, xq, wq);
    const std::vector<double> xn = gll_points(p);
    t.B.resize(n * n);
    t.D.resize(n * n);
    t.Gd.resize(n * n);
    for (int q = 0; q < n; ++q)
        for (int a = 0; a < n; ++a) {
            t.B[q * n + a] = lagrange(xn, a, xq[q]);
            t.Gd[q * n + a] = lagrange_d(xn, a, xq[q]);
            t.D[q * n + a] = lagrange_d(xq, a, xq[q]);
        }
    t.w = wq;
    t.geoV.assign(2 * 3 * n, 0.0);
    t.geoD.assign(2 * 3 * n, 0.0);
    t.geoVn.assign(2 * 3 * n, 0.0);
    for (int g = 1; g <= 2; ++g) {
        std::vector<double> xg(g + 1);
        for (int a = 0; a <= g; ++a) xg[a] = (double)a / g;
        for (int a = 0; a <= g; ++a)
            for (int q = 0; q < n; ++q) {
                t.geoV[(g - 1) * 3 * n + a * n + q] = lagrange(xg, a, xq[q]);
                t.geoD[(g - 1) * 3 * n + a * n + q] = lagrange_d(xg, a, xq[q]);
                t.geoVn[(g - 1) * 3 * n + a * n + q] = lagrange(xg, a, xn[q]);
            }
    }
    return t;
}

std::mutex g_upload_mu;
bool g_uploaded[64][HX_PMAX + 1];

cudaError_t ensure_tables(int device, int p) {
    std::lock_guard<std::mutex> lk(g_upload_mu);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (g_uploaded[device][p]) return cudaSuccess;
    Tables t = make_tables(p);
    for (int prec = 0; prec < 2; ++prec) {
        const hx::PrecOps *ops = hx::prec_ops(p, prec);
        cudaError_t e = ops->upload_tables(t.B.data(), t.D.data(), t.Gd.data(), t.w.data(), t.geoV.data(),
                                           t.geoD.data(), t.geoVn.data());
        if (e != cudaSuccess) return e;
        // the batch unit keeps its own copy of every degree's tables
        e = hx::batch_ops(prec)->upload_tables(p, t.B.data(), t.D.data(), t.Gd.data(), t.w.data(), t.geoV.data(),
                                               t.geoD.data(), t.geoVn.data());
        if (e != cudaSuccess) return e;
    }
    g_uploaded[device][p] = true;
    return cudaSuccess;
}

}  // namespace

// ---------------------------------------------------------------------------
// mesh object
// ---------------------------------------------------------------------------
struct QpCache {
    int storage = -1;
    bool valid = false;
    void *buf = nullptr;
    size_t bytes = 0;
};

struct hx_mesh {
    hx_ctx *ctx = nullptr;
    int p = 0, g = 1, n_elem = 0;
    int64_t n_nodes = 0, n_qp = 0, n_geo = 0;
    int64_t qs = 0;  // field stride of the SoA point arrays (n_qp rounded up to 32)
    int structured = 0, nx = 0, ny = 0, nz = 0;
    int law = 0;
    hx::MatParams mat{};
    int32_t *d_dof_conn = nullptr;
    uint8_t *d_dmask = nullptr;
    int64_t *d_cidx = nullptr;
    int64_t n_constrained = 0;
    double *d_geo_nodes = nullptr;
    int32_t *d_geo_conn = nullptr;
    double *d_geo64 = nullptr;
    float *d_geo32 = nullptr;
    double *d_fibH64 = nullptr;
    float *d_fibH32 = nullptr;
    double *d_fibM = nullptr;
    QpCache cache[2];
    int variant[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};  // autotuned apply variant per (prec, storage)
    int skip_stage_copies = 0;                // hx_set_wait_test
    int scatter_ordered = 0;                  // hx_set_scatter_mode
    void *w_elem[2] = {nullptr, nullptr};     // ordered assembly: element-local results per precision
    int64_t *d_gptr = nullptr, *d_gslot = nullptr;  // ordered assembly on a connectivity mesh: node -> slots
    long long wait_limit = 1ll << 32;        // cycles a bounded device wait polls
    // workspace (allocated on first use)
    std::vector<void *> ws;
    void *w_cheb_d[2] = {nullptr, nullptr}, *w_cheb_Kx[2] = {nullptr, nullptr};
    void *w_stage_in = nullptr, *w_stage_out = nullptr;
    // host-buffer apply in z-slabs: copy streams and events (created on first use)
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_start = nullptr, ev_out = nullptr, ev_in[8] = {}, ev_done[8] = {};
    std::vector<int64_t> h_cidx;  // the constrained DoFs, ascending (host copy of d_cidx)
    int host_slabs = 1;           // hx_set_host_apply_slabs: 0 whole vectors, 1 automatic, n at most n slabs
    double *w_cg = nullptr;   // r z zold p Ap dinv (FP64)
    double *w_newton = nullptr;  // Newton: residual, update, inverse diagonal (FP64)
    // host copies of the description (multigrid levels are rebuilt from them)
    std::vector<double> h_geo_nodes, h_frames;
    std::vector<int32_t> h_geo_conn;
    std::vector<uint8_t> h_dirichlet;
    hx_material h_mat{};
    float *w_cg32 = nullptr;  // r32 z32 dinv32
    cudaStream_t solve_stream = nullptr;
    hx::CgScalars *d_sc = nullptr;
    double *d_dots = nullptr, *d_partial = nullptr;
    double *h_pinned = nullptr;
};

namespace {

hx_status fail(hx_ctx *ctx, hx_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

hx_status cuda_fail(hx_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, HX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define HX_CUDA(ctx, call)                                           \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);   \
    } while (0)

// multiplier and shifts of the division by d >= 1 (see hx::FastDiv)
hx::FastDiv fast_div_of(int d) {
    const uint64_t dd = d > 0 ? (uint64_t)d : 1;
    int l = 0;
    while ((1ull << l) < dd) ++l;
    const uint64_t mm = (((1ull << 32) * ((1ull << l) - dd)) / dd) + 1;
    return hx::FastDiv{(uint32_t)mm, (uint32_t)(l < 1 ? l : 1), (uint32_t)(l > 1 ? l - 1 : 0)};
}

hx::MeshView view(const hx_mesh *m, int prec) {
    hx::MeshView v{};
    v.p = m->p;
    v.n_elem = m->n_elem;
    v.n_nodes = m->n_nodes;
    v.n_qp = m->n_qp;
    v.qs = m->qs;
    v.structured = m->structured;
    v.nx = m->nx;
    v.fnx = fast_div_of(m->nx);
    v.fny = fast_div_of(m->ny);
    v.ny = m->ny;
    v.nz = m->nz;
    v.Nx = (int64_t)m->nx * m->p + 1;
    v.Ny = (int64_t)m->ny * m->p + 1;
    v.dof_conn = m->d_dof_conn;
    v.geo = prec == HX_FP64 ? (const void *)m->d_geo64 : (const void *)m->d_geo32;
    v.geo64 = m->d_geo64;
    v.qp = m->cache[prec].buf;
    v.uk = m->cache[prec].buf;
    v.nf = m->cache[prec].storage >= 0 ? hx::qp_fields(m->law, m->cache[prec].storage) : 0;
    v.dmask = m->n_constrained ? m->d_dmask : nullptr;
    v.fibH = prec == HX_FP64 ? (const void *)m->d_fibH64 : (const void *)m->d_fibH32;
    v.fibH64 = m->d_fibH64;
    v.fibM = m->d_fibM;
    v.err = m->ctx->d_flags;
    v.mat = m->mat;
    v.matf = hx::MatParamsF{(float)m->mat.mu, (float)m->mat.lambda, (float)m->mat.kappa, (float)m->mat.k1,
                            (float)m->mat.k2};
    v.law = m->law;
    v.skip_stage_copies = m->skip_stage_copies;
    v.wait_limit = m->wait_limit;
    return v;
}

size_t prec_size(int prec) { return prec == HX_FP64 ? 8 : 4; }

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    return cudaMalloc((void **)p, n * sizeof(T) + HX_ARRAY_SLACK);  // bulk-copy windows may reach past the end
}

void dfree(void *p) {
    if (p) cudaFree(p);
}

bool bad_prec(int prec) { return prec != HX_FP64 && prec != HX_FP32; }

// Makes `device` current for the guard's lifetime and then makes the caller's
// previous device current again, so that no entry point leaves the calling
// thread switched to another device.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int device) {
        int cur = -1;
        err = cudaGetDevice(&cur);
        if (err == cudaSuccess && cur != device) {
            err = cudaSetDevice(device);
            if (err == cudaSuccess) prev = cur;
        }
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" {

hx_status hx_create(hx_ctx **ctx, int device, void *cuda_stream) {
    if (!ctx) return HX_ERR_ARG;
    *ctx = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) return HX_ERR_CUDA;
    DeviceGuard dg(device);
    if (dg.err != cudaSuccess) return HX_ERR_CUDA;
    hx_ctx *c = new hx_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    e = cudaMalloc((void **)&c->d_flags, 3 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_flags, 0, 3 * sizeof(int));
    if (e != cudaSuccess) {
        delete c;
        return HX_ERR_CUDA;
    }
    *ctx = c;
    return HX_OK;
}

void hx_destroy(hx_ctx *ctx) {
    if (!ctx) return;
    dfree(ctx->d_flags);
    delete ctx;
}

hx_status hx_set_stream(hx_ctx *ctx, void *cuda_stream) {
    if (!ctx) return HX_ERR_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return HX_OK;
}

const char *hx_last_error(hx_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

uint64_t hx_launch_count(hx_ctx *ctx, int32_t reset) {
    if (!ctx) return 0;
    const uint64_t v = ctx->launches;
    if (reset) ctx->launches = 0;
    return v;
}

hx_status hx_sync(hx_ctx *ctx, int timeout_ms) {
    if (!ctx) return HX_ERR_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaStreamQuery(ctx->stream);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_fail(ctx, q, "hx_sync");
        if (timeout_ms >= 0) {
            const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
            if (ms > timeout_ms) return fail(ctx, HX_ERR_TIMEOUT, "hx_sync: stream still busy after the time limit");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int flags[3] = {0, 0, 0};
    HX_CUDA(ctx, cudaMemcpy(flags, ctx->d_flags, sizeof flags, cudaMemcpyDeviceToHost));
    if (flags[0] || flags[1] || flags[2]) {
        HX_CUDA(ctx, cudaMemset(ctx->d_flags, 0, 3 * sizeof(int)));
        if (flags[2]) return fail(ctx, HX_ERR_TIMEOUT, "a kernel gave up waiting for staged quadrature-point data");
        if (flags[1]) return fail(ctx, HX_ERR_NAN, "NaN met in a quadrature-point state");
        return fail(ctx, HX_ERR_NONINVERTIBLE, "J <= 0 or det J0 <= 0 at a quadrature point");
    }
    return HX_OK;
}

hx_status hx_fibre_dispersion(double a, double b, double H[3]) {
    if (!H || !(a >= 0.0) || !(b > 0.0)) return HX_ERR_ARG;
    const double H33 = 1.0 / (4.0 * b) - std::exp(-2.0 * b) / (std::sqrt(2.0 * M_PI * b) * std::erf(std::sqrt(2.0 * b)));
    const double r = std::cyl_bessel_i(1.0, a) / std::cyl_bessel_i(0.0, a);
    H[0] = 0.5 * (1.0 - H33) * (1.0 + r);
    H[1] = 0.5 * (1.0 - H33) * (1.0 - r);
    H[2] = H33;
    return HX_OK;
}

// ---------------------------------------------------------------------------
// mesh setup
// ---------------------------------------------------------------------------
void hx_destroy_mesh(hx_mesh *m) {
    if (!m) return;
    cudaStreamSynchronize(m->ctx ? m->ctx->stream : nullptr);
    void *ptrs[] = {m->d_dof_conn, m->d_dmask, m->d_cidx, m->d_geo_nodes, m->d_geo_conn, m->d_geo64, m->d_geo32,
                    m->d_fibH64, m->d_fibH32, m->d_fibM, m->cache[0].buf, m->cache[1].buf, m->w_cheb_d[0],
                    m->w_cheb_d[1], m->w_cheb_Kx[0], m->w_cheb_Kx[1], m->w_stage_in, m->w_stage_out, m->w_cg, m->w_newton,
                    m->w_cg32, m->d_sc, m->d_dots, m->d_partial, m->w_elem[0], m->w_elem[1], m->d_gptr,
                    m->d_gslot};
    for (void *p : ptrs) dfree(p);
    if (m->h_pinned) cudaFreeHost(m->h_pinned);
    if (m->solve_stream) cudaStreamDestroy(m->solve_stream);
    for (cudaStream_t st : {m->s_h2d, m->s_d2h})
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : {m->ev_start, m->ev_out})
        if (ev) cudaEventDestroy(ev);
    for (int i = 0; i < 8; ++i) {
        if (m->ev_in[i]) cudaEventDestroy(m->ev_in[i]);
        if (m->ev_done[i]) cudaEventDestroy(m->ev_done[i]);
    }
    delete m;
}

hx_status hx_setup_mesh(hx_ctx *ctx, const hx_mesh_desc *d, const hx_material *mat, hx_mesh **out) {
    if (!ctx || !d || !mat || !out) return fail(ctx, HX_ERR_ARG, "hx_setup_mesh: null argument");
    *out = nullptr;
    if (d->p < HX_PMIN || d->p > HX_PMAX) return fail(ctx, HX_ERR_UNSUPPORTED, "hx_setup_mesh: degree outside 1..6");
    if (d->geo_degree != 1 && d->geo_degree != 2) return fail(ctx, HX_ERR_ARG, "hx_setup_mesh: geo_degree must be 1 or 2");
    if (d->n_elem < 0 || d->n_nodes <= 0 || d->n_geo_nodes <= 0 || !d->geo_nodes || !d->geo_conn)
        return fail(ctx, HX_ERR_ARG, "hx_setup_mesh: empty or missing geometry");
    if (mat->law < HX_CNH || mat->law > HX_FIBER) return fail(ctx, HX_ERR_ARG, "hx_setup_mesh: unknown law");
    if (mat->law == HX_FIBER && !d->fibre_frames && d->n_elem > 0)
        return fail(ctx, HX_ERR_ARG, "hx_setup_mesh: fibre law needs per-element fibre frames");
    const int p = d->p, n = p + 1, nq = n * n * n, g = d->geo_degree, ngg = (g + 1) * (g + 1) * (g + 1);
    int structured = 0;
    if (!d->dof_conn) {
        if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0 || (int64_t)d->nx * d->ny * d->nz != d->n_elem)
            return fail(ctx, HX_ERR_ARG, "hx_setup_mesh: structured box needs nx*ny*nz == n_elem");
        if (((int64_t)d->nx * p + 1) * ((int64_t)d->ny * p + 1) * ((int64_t)d->nz * p + 1) != d->n_nodes)
            return fail(ctx, HX_ERR_ARG, "hx_setup_mesh: n_nodes does not match the structured box");
        structured = 1;
    } else {
        for (int64_t i = 0; i < (int64_t)d->n_elem * nq; ++i)
            if (d->dof_conn[i] < 0 || d->dof_conn[i] >= d->n_nodes)
                return fail(ctx, HX_ERR_ARG, "hx_setup_mesh: dof_conn entry out of range");
    }
    for (int64_t i = 0; i < (int64_t)d->n_elem * ngg; ++i)
        if (d->geo_conn[i] < 0 || d->geo_conn[i] >= d->n_geo_nodes)
            return fail(ctx, HX_ERR_ARG, "hx_setup_mesh: geo_conn entry out of range");
    if ((int64_t)d->n_elem * nq >= ((int64_t)1 << 31) * 8)
        return fail(ctx, HX_ERR_ARG, "hx_setup_mesh: mesh too large");

    DeviceGuard dg(ctx->device);
    HX_CUDA(ctx, dg.err);
    HX_CUDA(ctx, ensure_tables(ctx->device, p));

    hx_mesh *m = new hx_mesh();
    m->ctx = ctx;
    m->p = p;
    m->g = g;
    m->n_elem = d->n_elem;
    m->n_nodes = d->n_nodes;
    m->n_qp = (int64_t)d->n_elem * nq;
    m->qs = (m->n_qp + 31) / 32 * 32;
    m->n_geo = d->n_geo_nodes;
    m->structured = structured;
    m->nx = d->nx;
    m->ny = d->ny;
    m->nz = d->nz;
    m->law = mat->law;
    m->mat = hx::MatParams{mat->mu, mat->lambda, mat->kappa, mat->k1, mat->k2};
    m->h_mat = *mat;
    m->h_geo_nodes.assign(d->geo_nodes, d->geo_nodes + 3 * d->n_geo_nodes);
    m->h_geo_conn.assign(d->geo_conn, d->geo_conn + (size_t)d->n_elem * ngg);
    if (d->fibre_frames && mat->law == HX_FIBER) m->h_frames.assign(d->fibre_frames, d->fibre_frames + 9 * (size_t)d->n_elem);
    if (d->dirichlet) m->h_dirichlet.assign(d->dirichlet, d->dirichlet + 3 * d->n_nodes);
    auto bail = [&](hx_status st) {
        hx_destroy_mesh(m);
        return st;
    };
#define HX_MCUDA(call)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return bail(cuda_fail(ctx, e_, #call));  \
    } while (0)
    cudaStream_t s = ctx->stream;
    const int64_t ne = d->n_elem;
    if (!structured && ne > 0) {
        HX_MCUDA(dalloc(&m->d_dof_conn, ne * nq));
        HX_MCUDA(cudaMemcpy(m->d_dof_conn, d->dof_conn, sizeof(int32_t) * ne * nq, cudaMemcpyHostToDevice));
    }
    HX_MCUDA(dalloc(&m->d_geo_nodes, 3 * d->n_geo_nodes));
    HX_MCUDA(cudaMemcpy(m->d_geo_nodes, d->geo_nodes, sizeof(double) * 3 * d->n_geo_nodes, cudaMemcpyHostToDevice));
    HX_MCUDA(dalloc(&m->d_geo_conn, ne * ngg));
    if (ne > 0)
        HX_MCUDA(cudaMemcpy(m->d_geo_conn, d->geo_conn, sizeof(int32_t) * ne * ngg, cudaMemcpyHostToDevice));
    // Dirichlet mask and the list of constrained DoFs
    if (d->dirichlet) {
        std::vector<int64_t> idx;
        for (int64_t i = 0; i < 3 * d->n_nodes; ++i)
            if (d->dirichlet[i]) idx.push_back(i);
        m->n_constrained = (int64_t)idx.size();
        if (m->n_constrained) {
            HX_MCUDA(dalloc(&m->d_dmask, 3 * d->n_nodes));
            HX_MCUDA(cudaMemcpy(m->d_dmask, d->dirichlet, 3 * d->n_nodes, cudaMemcpyHostToDevice));
            HX_MCUDA(dalloc(&m->d_cidx, idx.size()));
            HX_MCUDA(cudaMemcpy(m->d_cidx, idx.data(), sizeof(int64_t) * idx.size(), cudaMemcpyHostToDevice));
            m->h_cidx = idx;
        }
    }
    // fibre families per element: M1 and H_i = sum_k H_kk M_k (x) M_k (Sec. 3)
    {
        double Hd[3] = {0, 0, 0};
        if (mat->law == HX_FIBER) {
            if (hx_fibre_dispersion(mat->a, mat->b, Hd) != HX_OK)
                return bail(fail(ctx, HX_ERR_ARG, "hx_setup_mesh: invalid dispersion (a, b)"));
        }
        std::vector<double> fh(12 * (size_t)std::max<int64_t>(ne, 1), 0.0), fm(6 * (size_t)std::max<int64_t>(ne, 1), 0.0);
        std::vector<float> fh32(fh.size(), 0.0f);
        if (mat->law == HX_FIBER) {
            for (int64_t e = 0; e < ne; ++e) {
                const double *E1 = d->fibre_frames + 9 * e, *E2 = E1 + 3, *E3 = E1 + 6;
                for (int f = 0; f < 2; ++f) {
                    const double ph = f == 0 ? mat->phi : -mat->phi;
                    const double c = std::cos(ph), sn = std::sin(ph);
                    double M[3][3];
                    for (int k = 0; k < 3; ++k) {
                        M[0][k] = c * E1[k] + sn * E2[k];
                        M[1][k] = -sn * E1[k] + c * E2[k];
                        M[2][k] = E3[k];
                    }
                    const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
                    for (int k = 0; k < 6; ++k) {
                        const int i = pairs[k][0], j = pairs[k][1];
                        double v = 0.0;
                        for (int a = 0; a < 3; ++a) v += Hd[a] * M[a][i] * M[a][j];
                        fh[(size_t)(6 * f + k) * ne + e] = v;
                    }
                    for (int k = 0; k < 3; ++k) fm[(size_t)(3 * f + k) * ne + e] = M[0][k];
                }
            }
            for (size_t i = 0; i < fh.size(); ++i) fh32[i] = (float)fh[i];
        }
        HX_MCUDA(dalloc(&m->d_fibH64, fh.size()));
        HX_MCUDA(dalloc(&m->d_fibH32, fh.size()));
        HX_MCUDA(dalloc(&m->d_fibM, fm.size()));
        HX_MCUDA(cudaMemcpy(m->d_fibH64, fh.data(), sizeof(double) * fh.size(), cudaMemcpyHostToDevice));
        HX_MCUDA(cudaMemcpy(m->d_fibH32, fh32.data(), sizeof(float) * fh.size(), cudaMemcpyHostToDevice));
        HX_MCUDA(cudaMemcpy(m->d_fibM, fm.data(), sizeof(double) * fm.size(), cudaMemcpyHostToDevice));
    }
    // geometry at the quadrature points
    HX_MCUDA(dalloc(&m->d_geo64, 10 * (size_t)m->qs));
    HX_MCUDA(dalloc(&m->d_geo32, 10 * (size_t)m->qs));
    HX_MCUDA(cudaMemsetAsync(ctx->d_flags, 0, 3 * sizeof(int), s));
    {
        const hx::MeshView v = view(m, HX_FP64);
        HX_MCUDA(hx::prec_ops(p, HX_FP64)->geometry(v, m->d_geo_nodes, m->d_geo_conn, g, m->d_geo64, m->d_geo32, s));
        ctx->launches++;
    }
    HX_MCUDA(cudaStreamSynchronize(s));
    int flags[3];
    HX_MCUDA(cudaMemcpy(flags, ctx->d_flags, sizeof flags, cudaMemcpyDeviceToHost));
    if (flags[0]) {
        HX_MCUDA(cudaMemset(ctx->d_flags, 0, 3 * sizeof(int)));
        return bail(fail(ctx, HX_ERR_NONINVERTIBLE, "hx_setup_mesh: det J0 <= 0 at a quadrature point"));
    }
#undef HX_MCUDA
    *out = m;
    return HX_OK;
}

hx_status hx_mesh_info(const hx_mesh *m, int64_t *n_nodes, int64_t *n_elem, int64_t *n_qp) {
    if (!m) return HX_ERR_ARG;
    if (n_nodes) *n_nodes = m->n_nodes;
    if (n_elem) *n_elem = m->n_elem;
    if (n_qp) *n_qp = m->n_qp;
    return HX_OK;
}

hx_status hx_node_coords(hx_mesh *m, double *X_dev) {
    if (!m || !X_dev) return HX_ERR_ARG;
    hx_ctx *ctx = m->ctx;
    const hx::MeshView v = view(m, HX_FP64);
    HX_CUDA(ctx, hx::prec_ops(m->p, HX_FP64)->node_coords(v, m->d_geo_nodes, m->d_geo_conn, m->g, X_dev, ctx->stream));
    ctx->launches++;
    return HX_OK;
}

hx_status hx_apply_bytes(const hx_mesh *m, int32_t storage, int32_t prec, double *bytes) {
    if (!m || !bytes || bad_prec(prec) || storage < HX_RECOMPUTE || storage > HX_SPATIAL_TENSORS) return HX_ERR_ARG;
    const double s = (double)prec_size(prec);
    double b = 2.0 * 3.0 * m->n_nodes * s;    // read du, write out
    if (storage != HX_SPATIAL_TENSORS)
        b += 10.0 * m->n_qp * s;              // J0^-1, JxW (the spatial fields carry J_t^-1)
    if (storage == HX_RECOMPUTE)
        b += 3.0 * m->n_nodes * s;            // u_k
    else
        b += (double)hx::qp_fields(m->law, storage) * m->n_qp * s;
    if (!m->structured) b += 4.0 * m->n_qp;   // connectivity (one int per node slot)
    *bytes = b;
    return HX_OK;
}

// ---------------------------------------------------------------------------
// hot path
// ---------------------------------------------------------------------------
hx_status hx_precompute_qp(hx_mesh *m, const double *u_dev, int32_t store_prec, int32_t storage) {
    if (!m || !u_dev || bad_prec(store_prec) || storage < HX_RECOMPUTE || storage > HX_SPATIAL_TENSORS)
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_precompute_qp: bad argument");
    hx_ctx *ctx = m->ctx;
    QpCache &c = m->cache[store_prec];
    const size_t bytes = storage == HX_RECOMPUTE ? 3 * (size_t)m->n_nodes * prec_size(store_prec)
                                                 : (size_t)hx::qp_fields(m->law, storage) * m->qs * prec_size(store_prec);
    if (c.bytes != bytes) {
        dfree(c.buf);
        c.buf = nullptr;
        c.bytes = 0;
        HX_CUDA(ctx, cudaMalloc(&c.buf, bytes + HX_ARRAY_SLACK));  // bulk-copy windows may reach past the end
        c.bytes = bytes;
    }
    c.storage = storage;
    c.valid = false;
    const hx::MeshView v = view(m, store_prec);
    HX_CUDA(ctx, hx::prec_ops(m->p, store_prec)->precompute(v, storage, u_dev, c.buf, ctx->stream));
    ctx->launches += storage == HX_RECOMPUTE ? 2 : 1;
    c.valid = true;
    return HX_OK;
}

// Ordered assembly: the element buffer of `prec` (n_elem (p+1)^3 * 3 values),
// allocated on first use.
static hx_status ensure_elem_ws(hx_mesh *m, int prec) {
    if (!m->w_elem[prec])
        HX_CUDA(m->ctx, cudaMalloc(&m->w_elem[prec], 3 * (size_t)m->n_qp * prec_size(prec) + 64));
    return HX_OK;
}

// Operator kernels write their output either by atomic adds into the zeroed
// vector (default) or, in ordered mode, element by element into the element
// buffer, which gather_out then sums node by node in ascending element order.
static hx_status begin_out(hx_mesh *m, int prec, void *out, hx::MeshView &v) {
    hx_ctx *ctx = m->ctx;
    if (!m->scatter_ordered) {
        HX_CUDA(ctx, cudaMemsetAsync(out, 0, 3 * (size_t)m->n_nodes * prec_size(prec), ctx->stream));
        return HX_OK;
    }
    hx_status st = ensure_elem_ws(m, prec);
    if (st != HX_OK) return st;
    v.elem_out = m->w_elem[prec];
    return HX_OK;
}
static hx_status gather_out(hx_mesh *m, int prec, const hx::MeshView &v, void *out) {
    hx_ctx *ctx = m->ctx;
    if (!m->scatter_ordered) return HX_OK;
    if (m->structured)
        HX_CUDA(ctx, hx::gather_box(m->n_nodes, m->p, m->nx, m->ny, m->nz, m->w_elem[prec], v.dmask, out, prec,
                                    ctx->stream));
    else
        HX_CUDA(ctx, hx::gather_csr(m->n_nodes, m->d_gptr, m->d_gslot, m->w_elem[prec], v.dmask, out, prec,
                                    ctx->stream));
    ctx->launches++;
    return HX_OK;
}

static hx_status apply_dev(hx_mesh *m, const void *du, void *out, int prec) {
    hx_ctx *ctx = m->ctx;
    const QpCache &c = m->cache[prec];
    if (!c.valid) return fail(ctx, HX_ERR_NOT_READY, "hx_tangent_apply: no quadrature-point data at this precision (call hx_precompute_qp)");
    hx::MeshView v = view(m, prec);
    hx_status st = begin_out(m, prec, out, v);
    if (st != HX_OK) return st;
    HX_CUDA(ctx, hx::prec_ops(m->p, prec)->apply(v, c.storage, du, out, ctx->stream, m->variant[prec][c.storage]));
    ctx->launches++;
    st = gather_out(m, prec, v, out);
    if (st != HX_OK) return st;
    if (m->n_constrained) {
        HX_CUDA(ctx, hx::copy_idx(m->d_cidx, m->n_constrained, du, out, prec, ctx->stream));
        ctx->launches++;
    }
    return HX_OK;
}

hx_status hx_tangent_apply(hx_mesh *m, const void *du_dev, void *out_dev, int32_t prec) {
    if (!m || !du_dev || !out_dev || bad_prec(prec) || du_dev == out_dev)
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_tangent_apply: bad argument");
    return apply_dev(m, du_dev, out_dev, prec);
}

hx_status hx_set_host_apply_slabs(hx_mesh *m, int32_t slabs) {
    if (!m || slabs < 0 || slabs > 8) return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_set_host_apply_slabs: bad argument");
    m->host_slabs = slabs;
    return HX_OK;
}

hx_status hx_set_scatter_mode(hx_mesh *m, int32_t mode) {
    if (!m || (mode != HX_SCATTER_ATOMIC && mode != HX_SCATTER_ORDERED))
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_set_scatter_mode: bad argument");
    hx_ctx *ctx = m->ctx;
    if (mode == HX_SCATTER_ORDERED && !m->structured && !m->d_gptr) {
        // node -> (element, local node) slots, ascending in element and local node
        const int64_t nq = (int64_t)(m->p + 1) * (m->p + 1) * (m->p + 1);
        std::vector<int32_t> conn((size_t)(m->n_elem * nq));
        HX_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        HX_CUDA(ctx, cudaMemcpy(conn.data(), m->d_dof_conn, conn.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
        std::vector<int64_t> ptr((size_t)m->n_nodes + 1, 0), slot(conn.size());
        for (int32_t v : conn) ptr[(size_t)v + 1]++;
        for (int64_t i = 0; i < m->n_nodes; ++i) ptr[(size_t)i + 1] += ptr[(size_t)i];
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t s = 0; s < (int64_t)conn.size(); ++s) slot[(size_t)fill[(size_t)conn[(size_t)s]]++] = s;
        HX_CUDA(ctx, cudaMalloc((void **)&m->d_gptr, ptr.size() * sizeof(int64_t)));
        HX_CUDA(ctx, cudaMalloc((void **)&m->d_gslot, (slot.size() + 1) * sizeof(int64_t)));
        HX_CUDA(ctx, cudaMemcpy(m->d_gptr, ptr.data(), ptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
        HX_CUDA(ctx, cudaMemcpy(m->d_gslot, slot.data(), slot.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    }
    m->scatter_ordered = mode == HX_SCATTER_ORDERED;
    return HX_OK;
}

hx_status hx_set_wait_test(hx_mesh *m, int32_t skip_stage_copies, int64_t wait_limit_cycles) {
    if (!m || wait_limit_cycles < 0) return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_set_wait_test: bad argument");
    m->skip_stage_copies = skip_stage_copies ? 1 : 0;
    m->wait_limit = wait_limit_cycles ? (long long)wait_limit_cycles : (1ll << 32);
    return HX_OK;
}

hx_status hx_set_apply_variant(hx_mesh *m, int32_t prec, int32_t storage, int32_t variant) {
    if (!m || bad_prec(prec) || storage < HX_RECOMPUTE || storage > HX_SPATIAL_TENSORS || variant < 0 ||
        variant >= hx::prec_ops(m->p, prec)->n_variants)
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_set_apply_variant: bad argument");
    m->variant[prec][storage] = variant;
    return HX_OK;
}

hx_status hx_autotune(hx_mesh *m, int32_t prec, const void *du_dev, void *out_dev, int32_t reps, int32_t *best_variant,
                      double times_ms[6]) {
    if (!m || bad_prec(prec) || !du_dev || !out_dev || du_dev == out_dev || reps < 1)
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_autotune: bad argument");
    hx_ctx *ctx = m->ctx;
    const QpCache &c = m->cache[prec];
    if (!c.valid) return fail(ctx, HX_ERR_NOT_READY, "hx_autotune: no quadrature-point data at this precision");
    const hx::PrecOps *ops = hx::prec_ops(m->p, prec);
    const hx::MeshView v = view(m, prec);
    cudaEvent_t a, b;
    HX_CUDA(ctx, cudaEventCreate(&a));
    HX_CUDA(ctx, cudaEventCreate(&b));
    int best = 0;
    double tbest = 1e30, t[8];
    for (int var = 0; var < ops->n_variants && var < 8; ++var) {
        cudaError_t e = ops->apply(v, c.storage, du_dev, out_dev, ctx->stream, var);  // warm-up
        if (e != cudaSuccess) {
            cudaGetLastError();
            t[var] = -1.0;
            continue;
        }
        cudaEventRecord(a, ctx->stream);
        for (int r = 0; r < reps; ++r) ops->apply(v, c.storage, du_dev, out_dev, ctx->stream, var);
        cudaEventRecord(b, ctx->stream);
        e = cudaEventSynchronize(b);
        if (e != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return cuda_fail(ctx, e, "hx_autotune");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        t[var] = ms / reps;
        ctx->launches += reps + 1;
        if (t[var] < tbest) {
            tbest = t[var];
            best = var;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    m->variant[prec][c.storage] = best;
    if (best_variant) *best_variant = best;
    if (times_ms)
        for (int i = 0; i < 6; ++i) times_ms[i] = i < ops->n_variants ? t[i] : -1.0;
    return HX_OK;
}

// The mesh view of the element layers z0 <= ez < z1 of a structured box: the
// point arrays start at the slab's first point and the node-indexed arrays at
// its first node layer (z0 p), so the kernels run on the slab as on a box of
// z1 - z0 layers. Vectors passed with it must be offset by the same node
// layer. Not for the fibre law (its per-element arrays are strided by the
// element count) nor for ordered assembly.
// slabs of the host-buffer apply unless the mesh sets its own limit
constexpr int HX_HOST_SLABS = 4;

hx::MeshView slab_view(const hx_mesh *m, int prec, int z0, int z1) {
    hx::MeshView v = view(m, prec);
    const size_t sz = prec_size(prec);
    const int64_t nq = (int64_t)(m->p + 1) * (m->p + 1) * (m->p + 1);
    const int64_t e0 = (int64_t)z0 * m->nx * m->ny;
    const int64_t node0 = (int64_t)z0 * m->p * v.Nx * v.Ny;
    v.n_elem = (z1 - z0) * m->nx * m->ny;
    v.nz = z1 - z0;
    v.n_nodes = v.Nx * v.Ny * ((int64_t)(z1 - z0) * m->p + 1);
    v.n_qp = (int64_t)v.n_elem * nq;
    v.geo = (const char *)v.geo + e0 * nq * sz;
    v.geo64 = v.geo64 + e0 * nq;
    v.qp = (const char *)v.qp + e0 * nq * sz;  // point-indexed caches
    v.uk = (const char *)v.uk + 3 * node0 * sz;  // the recompute strategy's node vector u_k
    if (v.dmask) v.dmask += 3 * node0;
    return v;
}

// out = K(u_k) du from host vectors on a structured box, in z-slabs of element
// layers on three streams: the copy of slab s + 1's node layers to the device
// overlaps the apply of slab s, and the node layers that no later slab touches
// are fixed on constrained rows and copied back while the next slabs run.
// Sets *done = false, doing nothing, where it does not apply (connectivity
// meshes, the fibre law, ordered assembly, fewer than four element layers, or
// no slab split whose point chunks start on 16-byte boundaries).
hx_status apply_host_slabs(hx_mesh *m, const void *du_host, void *out_host, int prec, bool *done) {
    *done = false;
    hx_ctx *ctx = m->ctx;
    const QpCache &c = m->cache[prec];
    if (!m->structured || m->scatter_ordered || m->law == HX_FIBER || !c.valid || m->nz < 4) return HX_OK;
    const size_t sz = prec_size(prec);
    const int64_t nq = (int64_t)(m->p + 1) * (m->p + 1) * (m->p + 1);
    const int64_t lay = (int64_t)m->nx * m->ny;
    int k = 0;  // element layers per slab
    const int most = m->host_slabs >= 2 ? m->host_slabs : HX_HOST_SLABS;
    for (int ns = std::min(most, m->nz / 2); ns >= 2 && !k; --ns) {
        const int kk = (m->nz + ns - 1) / ns;
        bool ok = true;
        for (int z0 = kk; z0 < m->nz; z0 += kk) ok = ok && ((int64_t)z0 * lay * nq * (int64_t)sz) % 16 == 0;
        if (ok) k = kk;
    }
    if (!k) return HX_OK;
    if (!m->s_h2d) {
        DeviceGuard dg(ctx->device);
        HX_CUDA(ctx, cudaStreamCreateWithFlags(&m->s_h2d, cudaStreamNonBlocking));
        HX_CUDA(ctx, cudaStreamCreateWithFlags(&m->s_d2h, cudaStreamNonBlocking));
        HX_CUDA(ctx, cudaEventCreateWithFlags(&m->ev_start, cudaEventDisableTiming));
        HX_CUDA(ctx, cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming));
        for (int i = 0; i < 8; ++i) {
            HX_CUDA(ctx, cudaEventCreateWithFlags(&m->ev_in[i], cudaEventDisableTiming));
            HX_CUDA(ctx, cudaEventCreateWithFlags(&m->ev_done[i], cudaEventDisableTiming));
        }
    }
    const int64_t Nx = (int64_t)m->nx * m->p + 1, Ny = (int64_t)m->ny * m->p + 1;
    const int64_t Nz = (int64_t)m->nz * m->p + 1;
    const int64_t lv = 3 * Nx * Ny;  // values per node layer
    const char *hin = (const char *)du_host;
    char *hout = (char *)out_host;
    char *din = (char *)m->w_stage_in, *dout = (char *)m->w_stage_out;
    const int variant = m->variant[prec][c.storage];
    HX_CUDA(ctx, cudaEventRecord(m->ev_start, ctx->stream));
    HX_CUDA(ctx, cudaStreamWaitEvent(m->s_h2d, m->ev_start, 0));
    HX_CUDA(ctx, cudaStreamWaitEvent(m->s_d2h, m->ev_start, 0));
    HX_CUDA(ctx, cudaMemsetAsync(dout, 0, (size_t)(lv * Nz) * sz, ctx->stream));
    int64_t in_done = 0, out_done = 0;  // node layers copied in and out so far
    for (int z0 = 0, s = 0; z0 < m->nz; z0 += k, ++s) {
        const int z1 = std::min(z0 + k, m->nz);
        const int64_t need = (int64_t)z1 * m->p + 1;  // node layers this slab reads
        HX_CUDA(ctx, cudaMemcpyAsync(din + in_done * lv * sz, hin + in_done * lv * sz, (size_t)((need - in_done) * lv) * sz,
                                     cudaMemcpyHostToDevice, m->s_h2d));
        in_done = need;
        HX_CUDA(ctx, cudaEventRecord(m->ev_in[s], m->s_h2d));
        HX_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, m->ev_in[s], 0));
        const hx::MeshView v = slab_view(m, prec, z0, z1);
        const int64_t off = (int64_t)z0 * m->p * lv;
        HX_CUDA(ctx, hx::prec_ops(m->p, prec)->apply(v, c.storage, din + off * sz, dout + off * sz, ctx->stream, variant));
        ctx->launches++;
        HX_CUDA(ctx, cudaEventRecord(m->ev_done[s], ctx->stream));
        HX_CUDA(ctx, cudaStreamWaitEvent(m->s_d2h, m->ev_done[s], 0));
        const int64_t ready = z1 == m->nz ? Nz : (int64_t)z1 * m->p;  // node layers no later slab touches
        if (m->n_constrained) {  // constrained rows: out = du
            const auto lo = std::lower_bound(m->h_cidx.begin(), m->h_cidx.end(), out_done * lv);
            const auto hi = std::lower_bound(m->h_cidx.begin(), m->h_cidx.end(), ready * lv);
            if (hi > lo) {
                HX_CUDA(ctx, hx::copy_idx(m->d_cidx + (lo - m->h_cidx.begin()), hi - lo, din, dout, prec, m->s_d2h));
                ctx->launches++;
            }
        }
        HX_CUDA(ctx, cudaMemcpyAsync(hout + out_done * lv * sz, dout + out_done * lv * sz,
                                     (size_t)((ready - out_done) * lv) * sz, cudaMemcpyDeviceToHost, m->s_d2h));
        out_done = ready;
    }
    HX_CUDA(ctx, cudaEventRecord(m->ev_out, m->s_d2h));
    HX_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, m->ev_out, 0));
    HX_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *done = true;
    return HX_OK;
}

hx_status hx_tangent_apply_host(hx_mesh *m, const void *du_host, void *out_host, int32_t prec) {
    if (!m || !du_host || !out_host || bad_prec(prec))
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_tangent_apply_host: bad argument");
    hx_ctx *ctx = m->ctx;
    const size_t bytes = 3 * (size_t)m->n_nodes * prec_size(prec);
    if (!m->w_stage_in) {
        HX_CUDA(ctx, cudaMalloc(&m->w_stage_in, 3 * (size_t)m->n_nodes * 8 + 16));
        HX_CUDA(ctx, cudaMalloc(&m->w_stage_out, 3 * (size_t)m->n_nodes * 8 + 16));
    }
    if (m->host_slabs) {
        bool done = false;
        const hx_status st = apply_host_slabs(m, du_host, out_host, prec, &done);
        if (st != HX_OK || done) return st;
    }
    HX_CUDA(ctx, cudaMemcpyAsync(m->w_stage_in, du_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    hx_status st = apply_dev(m, m->w_stage_in, m->w_stage_out, prec);
    if (st != HX_OK) return st;
    HX_CUDA(ctx, cudaMemcpyAsync(out_host, m->w_stage_out, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    HX_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HX_OK;
}

hx_status hx_residual(hx_mesh *m, const void *u_dev, void *r_dev, int32_t prec) {
    if (!m || !u_dev || !r_dev || bad_prec(prec) || u_dev == r_dev)
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_residual: bad argument");
    hx_ctx *ctx = m->ctx;
    hx::MeshView v = view(m, prec);
    hx_status st = begin_out(m, prec, r_dev, v);
    if (st != HX_OK) return st;
    HX_CUDA(ctx, hx::prec_ops(m->p, prec)->residual(v, u_dev, r_dev, ctx->stream));
    ctx->launches++;
    return gather_out(m, prec, v, r_dev);
}

hx_status hx_diagonal(hx_mesh *m, void *diag_dev, int32_t prec) {
    if (!m || !diag_dev || bad_prec(prec)) return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_diagonal: bad argument");
    hx_ctx *ctx = m->ctx;
    const QpCache &c = m->cache[prec];
    if (!c.valid) return fail(ctx, HX_ERR_NOT_READY, "hx_diagonal: no quadrature-point data at this precision");
    hx::MeshView v = view(m, prec);
    hx_status st = begin_out(m, prec, diag_dev, v);
    if (st != HX_OK) return st;
    HX_CUDA(ctx, hx::prec_ops(m->p, prec)->diagonal(v, c.storage, diag_dev, ctx->stream));
    ctx->launches++;
    st = gather_out(m, prec, v, diag_dev);
    if (st != HX_OK) return st;
    if (m->n_constrained) {
        HX_CUDA(ctx, hx::set_idx(m->d_cidx, m->n_constrained, 1.0, diag_dev, prec, ctx->stream));
        ctx->launches++;
    }
    return HX_OK;
}

static hx_status ensure_cheb_ws(hx_mesh *m, int prec) {
    if (!m->w_cheb_d[prec]) {
        const size_t b = 3 * (size_t)m->n_nodes * prec_size(prec) + 16;
        HX_CUDA(m->ctx, cudaMalloc(&m->w_cheb_d[prec], b));
        HX_CUDA(m->ctx, cudaMalloc(&m->w_cheb_Kx[prec], b));
    }
    return HX_OK;
}

static hx_status cheb_run(hx_mesh *m, const void *rhs, void *x, const void *dinv, int degree, double lmax,
                          double range, int zero_initial, int prec) {
    hx_ctx *ctx = m->ctx;
    hx_status st = ensure_cheb_ws(m, prec);
    if (st != HX_OK) return st;
    const double a = lmax / range, b = lmax;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a);
    const int64_t n = 3 * m->n_nodes;
    double rho_prev = 0.0;
    for (int k = 0; k < degree; ++k) {
        const void *Kx = nullptr;
        if (!(k == 0 && zero_initial)) {
            st = apply_dev(m, x, m->w_cheb_Kx[prec], prec);
            if (st != HX_OK) return st;
            Kx = m->w_cheb_Kx[prec];
        }
        double cd, cr, rho;
        if (k == 0) {
            rho = delta / theta;
            cd = 0.0;
            cr = 1.0 / theta;
        } else {
            rho = 1.0 / (2.0 * theta / delta - rho_prev);
            cd = rho * rho_prev;
            cr = 2.0 * rho / delta;
        }
        HX_CUDA(ctx, hx::cheb_update(n, rhs, Kx, dinv, m->w_cheb_d[prec], x, cd, cr, k == 0, prec, ctx->stream));
        ctx->launches++;
        rho_prev = rho;
    }
    return HX_OK;
}

hx_status hx_chebyshev_smooth(hx_mesh *m, const void *rhs_dev, void *x_dev, const void *inv_diag_dev, int32_t degree,
                              double lambda_max, double smoothing_range, int32_t zero_initial, int32_t prec) {
    if (!m || !rhs_dev || !x_dev || !inv_diag_dev || bad_prec(prec) || degree < 0 || !(lambda_max > 0.0) ||
        !(smoothing_range > 1.0))
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_chebyshev_smooth: bad argument");
    return cheb_run(m, rhs_dev, x_dev, inv_diag_dev, degree, lambda_max, smoothing_range, zero_initial, prec);
}

// ---------------------------------------------------------------------------
// Chebyshev-Jacobi smoother without allocation
//
// Some callers cannot allocate device memory once they are running: a solver
// embedded in an application whose memory is fully reserved by another
// framework's caching allocator (where cudaMalloc fails or must not be used),
// or a latency-critical loop in which cudaMalloc/cudaFree would synchronise the
// device and stall other streams. For them the two scratch vectors of the
// smoother (the Chebyshev update d and the operator product K x) live in the
// file-scope device array below instead of mesh-owned workspace.
//
// Limit: HX_NOALLOC_MAX_DOFS DoFs per vector (1,048,576, i.e. 349,525 nodes);
// the array holds 2 * HX_NOALLOC_MAX_DOFS doubles (16 MiB) on every GPU that
// loads the library, until the process exits.
// ---------------------------------------------------------------------------
#define HX_NOALLOC_MAX_DOFS (1 << 20)
static __device__ __align__(256) double g_noalloc_scratch[2 * HX_NOALLOC_MAX_DOFS];
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];  // device address of the array, per device

// Device address of the scratch array on the context's device. In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) with cudaGetSymbolAddress.
static hx_status noalloc_scratch(hx_ctx *ctx, void **addr) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (ctx->device < 0 || ctx->device >= 64) return fail(ctx, HX_ERR_ARG, "noalloc: device index out of range");
    if (!g_noalloc_addr[ctx->device]) {
        DeviceGuard dg(ctx->device);  // the caller's current device is restored on return
        HX_CUDA(ctx, dg.err);
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[ctx->device] = p;
    }
    *addr = g_noalloc_addr[ctx->device];
    return HX_OK;
}

extern "C" hx_status hx_chebyshev_smooth_noalloc(hx_mesh *m, const void *rhs_dev, void *x_dev,
                                                 const void *inv_diag_dev, int32_t degree, double lambda_max,
                                                 double smoothing_range, int32_t zero_initial, int32_t prec) {
    if (!m || !rhs_dev || !x_dev || !inv_diag_dev || bad_prec(prec) || degree < 0 || !(lambda_max > 0.0) ||
        !(smoothing_range > 1.0))
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_chebyshev_smooth_noalloc: bad argument");
    hx_ctx *ctx = m->ctx;
    const int64_t n = 3 * m->n_nodes;
    if (n > HX_NOALLOC_MAX_DOFS)
        return fail(ctx, HX_ERR_ARG,
                    "hx_chebyshev_smooth_noalloc: mesh has " + std::to_string(n) + " DoFs, more than the " +
                        std::to_string(HX_NOALLOC_MAX_DOFS) + " the static scratch array holds");
    void *base = nullptr;
    hx_status st = noalloc_scratch(ctx, &base);
    if (st != HX_OK) return st;
    void *d = base;                                              // Chebyshev update d
    void *Kx = (void *)((double *)base + HX_NOALLOC_MAX_DOFS);   // operator product K x
    const double a = lambda_max / smoothing_range, b = lambda_max;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a);
    double rho_prev = 0.0;
    for (int k = 0; k < degree; ++k) {
        const void *kx = nullptr;
        if (!(k == 0 && zero_initial)) {
            st = apply_dev(m, x_dev, Kx, prec);  // zeroes Kx itself before accumulating
            if (st != HX_OK) return st;
            kx = Kx;
        }
        double cd, cr, rho;
        if (k == 0) {  // the first step overwrites d, so the array's old contents never leak in
            rho = delta / theta;
            cd = 0.0;
            cr = 1.0 / theta;
        } else {
            rho = 1.0 / (2.0 * theta / delta - rho_prev);
            cd = rho * rho_prev;
            cr = 2.0 * rho / delta;
        }
        HX_CUDA(ctx, hx::cheb_update(n, rhs_dev, kx, inv_diag_dev, d, x_dev, cd, cr, k == 0, prec, ctx->stream));
        ctx->launches++;
        rho_prev = rho;
    }
    return HX_OK;
}

static hx_status ensure_cg_ws(hx_mesh *m) {
    hx_ctx *ctx = m->ctx;
    if (m->w_cg) return HX_OK;
    const size_t n = 3 * (size_t)m->n_nodes;
    HX_CUDA(ctx, cudaMalloc((void **)&m->w_cg, 6 * n * sizeof(double) + 64));
    HX_CUDA(ctx, cudaMalloc((void **)&m->w_cg32, 3 * n * sizeof(float) + 64));
    HX_CUDA(ctx, cudaMalloc((void **)&m->d_sc, sizeof(hx::CgScalars)));
    HX_CUDA(ctx, cudaMalloc((void **)&m->d_dots, 8 * sizeof(double)));
    HX_CUDA(ctx, cudaMalloc((void **)&m->d_partial, 3 * hx::RED_BLOCKS * sizeof(double)));
    HX_CUDA(ctx, cudaHostAlloc((void **)&m->h_pinned, 8 * sizeof(double), cudaHostAllocDefault));
    return HX_OK;
}

hx_status hx_estimate_lambda_max(hx_mesh *m, const double *inv_diag_dev, int32_t iters, uint64_t seed, double *out) {
    if (!m || !inv_diag_dev || !out || iters < 1) return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_estimate_lambda_max: bad argument");
    hx_ctx *ctx = m->ctx;
    hx_status st = ensure_cg_ws(m);
    if (st != HX_OK) return st;
    const int64_t n = 3 * m->n_nodes;
    double *v = m->w_cg, *y = m->w_cg + n, *w = m->w_cg + 2 * n;
    cudaStream_t s = ctx->stream;
    HX_CUDA(ctx, hx::random_vec(n, seed, w, s));
    HX_CUDA(ctx, hx::dots(n, 1, w, w, nullptr, nullptr, nullptr, nullptr, m->d_partial, m->d_dots, s));
    HX_CUDA(ctx, hx::normalize(n, m->d_dots, w, v, s));
    for (int it = 0; it < iters; ++it) {
        st = apply_dev(m, v, y, HX_FP64);
        if (st != HX_OK) return st;
        HX_CUDA(ctx, hx::scale(n, inv_diag_dev, y, w, s));
        HX_CUDA(ctx, hx::dots(n, 1, w, w, nullptr, nullptr, nullptr, nullptr, m->d_partial, m->d_dots, s));
        HX_CUDA(ctx, hx::normalize(n, m->d_dots, w, v, s));
        ctx->launches += 5;
    }
    double nrm2 = 0.0;
    HX_CUDA(ctx, cudaMemcpyAsync(&nrm2, m->d_dots, sizeof(double), cudaMemcpyDeviceToHost, s));
    HX_CUDA(ctx, cudaStreamSynchronize(s));
    *out = std::sqrt(nrm2);
    return HX_OK;
}

// Preconditioner z = M r: Chebyshev(degree)-Jacobi from zero in precision pp
// (degree 0 = plain Jacobi), FP64 in and out.
static hx_status cg_precond(hx_mesh *m, int pp, int degree, double lmax, double range, const double *r, double *z,
                            const void *dinv, bool r32_ready) {
    hx_ctx *ctx = m->ctx;
    const int64_t n = 3 * m->n_nodes;
    cudaStream_t s = ctx->stream;
    float *r32 = m->w_cg32, *z32 = m->w_cg32 + n;
    if (pp == HX_FP32) {
        if (!r32_ready) HX_CUDA(ctx, hx::to_f32(n, r, r32, s));
        if (degree == 0) {
            HX_CUDA(ctx, hx::cheb_update(n, r32, nullptr, dinv, m->w_cheb_d[pp], z32, 0.0, 1.0, 1, pp, s));
        } else {
            hx_status st = cheb_run(m, r32, z32, dinv, degree, lmax, range, 1, pp);
            if (st != HX_OK) return st;
        }
        HX_CUDA(ctx, hx::to_f64(n, z32, z, s));
        ctx->launches += 2;
    } else {
        if (degree == 0) {
            HX_CUDA(ctx, hx::cheb_update(n, r, nullptr, dinv, m->w_cheb_d[pp], z, 0.0, 1.0, 1, pp, s));
        } else {
            hx_status st = cheb_run(m, r, z, dinv, degree, lmax, range, 1, pp);
            if (st != HX_OK) return st;
        }
    }
    return HX_OK;
}

// Flexible (Polak-Ribiere) CG in FP64 on the mesh's constrained tangent with
// the preconditioner z = M r given by `prec_setup` (run once, on the solve
// stream) and `precond` (r in FP64, and in FP32 in w_cg32 when r32_ready).
typedef std::function<hx_status(const double *r, double *z, bool r32_ready)> PrecondFn;
static hx_status cg_core(hx_mesh *m, const double *rhs, double *x, double tol, int32_t max_iter, int pp, int use_graph,
                         const std::function<hx_status()> &prec_setup, const PrecondFn &precond, int32_t *iters,
                         double *rel_residual) {
    hx_ctx *ctx = m->ctx;
    hx_status st = ensure_cg_ws(m);
    if (st != HX_OK) return st;
    if (!m->solve_stream) HX_CUDA(ctx, cudaStreamCreateWithFlags(&m->solve_stream, cudaStreamNonBlocking));
    // run the solve on a private (capturable) stream ordered after the caller's stream
    cudaStream_t user = ctx->stream;
    cudaEvent_t ev;
    HX_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    HX_CUDA(ctx, cudaEventRecord(ev, user));
    HX_CUDA(ctx, cudaStreamWaitEvent(m->solve_stream, ev, 0));
    ctx->stream = m->solve_stream;
    struct Restore {
        hx_ctx *c;
        cudaStream_t u;
        cudaEvent_t e;
        ~Restore() {
            cudaEventRecord(e, c->stream);
            cudaStreamWaitEvent(u, e, 0);
            c->stream = u;
            cudaEventDestroy(e);
        }
    } restore{ctx, user, ev};
    cudaStream_t s = ctx->stream;

    const int64_t n = 3 * m->n_nodes;
    double *r = m->w_cg, *z = r + n, *zold = r + 2 * n, *p = r + 3 * n, *Ap = r + 4 * n;
    st = prec_setup();
    if (st != HX_OK) return st;
    // r = b - K x ; z = M r ; p = zold = z
    st = apply_dev(m, x, Ap, HX_FP64);
    if (st != HX_OK) return st;
    HX_CUDA(ctx, hx::sub(n, rhs, Ap, r, s));
    st = precond(r, z, false);
    if (st != HX_OK) return st;
    HX_CUDA(ctx, cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    HX_CUDA(ctx, cudaMemcpyAsync(zold, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    HX_CUDA(ctx, hx::dots(n, 3, r, z, r, r, rhs, rhs, m->d_partial, m->d_dots, s));
    double h3[3];
    HX_CUDA(ctx, cudaMemcpyAsync(h3, m->d_dots, sizeof h3, cudaMemcpyDeviceToHost, s));
    HX_CUDA(ctx, cudaStreamSynchronize(s));
    const double bnorm = std::sqrt(h3[2]);
    hx::CgScalars sc0{};
    sc0.rz = h3[0];
    sc0.rr = h3[1];
    HX_CUDA(ctx, cudaMemcpyAsync(m->d_sc, &sc0, sizeof sc0, cudaMemcpyHostToDevice, s));
    HX_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->launches += 8;
    if (bnorm == 0.0) {
        HX_CUDA(ctx, cudaMemsetAsync(x, 0, n * sizeof(double), s));
        if (iters) *iters = 0;
        if (rel_residual) *rel_residual = 0.0;
        return HX_OK;
    }

    auto body = [&]() -> hx_status {
        hx_status b = apply_dev(m, p, Ap, HX_FP64);
        if (b != HX_OK) return b;
        HX_CUDA(ctx, hx::dots(n, 1, p, Ap, nullptr, nullptr, nullptr, nullptr, m->d_partial, &m->d_sc->pAp, s));
        HX_CUDA(ctx, hx::cg_alpha(m->d_sc, s));
        HX_CUDA(ctx, hx::cg_xr(n, m->d_sc, p, Ap, x, r, pp == HX_FP32 ? m->w_cg32 : nullptr, s));
        b = precond(r, z, true);
        if (b != HX_OK) return b;
        HX_CUDA(ctx, hx::dots(n, 3, r, z, r, zold, r, r, m->d_partial, m->d_dots, s));
        HX_CUDA(ctx, hx::cg_beta(m->d_sc, m->d_dots, s));
        HX_CUDA(ctx, hx::cg_p(n, m->d_sc, z, p, zold, s));
        HX_CUDA(ctx, cudaMemcpyAsync(m->h_pinned, m->d_sc, sizeof(hx::CgScalars), cudaMemcpyDeviceToHost, s));
        ctx->launches += 8;
        return HX_OK;
    };

    cudaGraphExec_t exec = nullptr;
    if (use_graph) {
        cudaGraph_t graph = nullptr;
        HX_CUDA(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        hx_status b = body();
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (b != HX_OK) {
            if (graph) cudaGraphDestroy(graph);
            return b;
        }
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaGraphInstantiate");
    }
    struct ExecGuard {
        cudaGraphExec_t e;
        ~ExecGuard() {
            if (e) cudaGraphExecDestroy(e);
        }
    } eg{exec};
    int it = 0;
    double rel = std::sqrt(sc0.rr) / bnorm;
    bool bad = false;
    while (it < max_iter && rel > tol) {
        if (exec) {
            HX_CUDA(ctx, cudaGraphLaunch(exec, s));
            ctx->launches += 8;
        } else {
            st = body();
            if (st != HX_OK) return st;
        }
        HX_CUDA(ctx, cudaStreamSynchronize(s));
        const hx::CgScalars *hs = (const hx::CgScalars *)m->h_pinned;
        ++it;
        if (hs->bad) {
            bad = true;
            break;
        }
        rel = std::sqrt(hs->rr) / bnorm;
    }
    // true residual at exit
    st = apply_dev(m, x, Ap, HX_FP64);
    if (st != HX_OK) return st;
    HX_CUDA(ctx, hx::sub(n, rhs, Ap, r, s));
    HX_CUDA(ctx, hx::dots(n, 1, r, r, nullptr, nullptr, nullptr, nullptr, m->d_partial, m->d_dots, s));
    double rr = 0.0;
    HX_CUDA(ctx, cudaMemcpyAsync(&rr, m->d_dots, sizeof rr, cudaMemcpyDeviceToHost, s));
    HX_CUDA(ctx, cudaStreamSynchronize(s));
    const double true_rel = std::sqrt(rr) / bnorm;
    if (iters) *iters = it;
    if (rel_residual) *rel_residual = true_rel;
    if (bad || !(true_rel == true_rel))
        return fail(ctx, HX_ERR_NAN, "CG breakdown (NaN or non-positive curvature p.Kp <= 0) at iteration " +
                                         std::to_string(it));
    if (true_rel > tol) return fail(ctx, HX_ERR_NOT_CONVERGED, "CG tolerance not reached");
    return HX_OK;
}

hx_status hx_cg_solve(hx_mesh *m, const double *rhs, double *x, double tol, int32_t max_iter, const hx_cg_options *opt,
                      int32_t *iters, double *rel_residual) {
    if (!m || !rhs || !x || !opt || max_iter < 0 || !(tol > 0.0) || bad_prec(opt->precond_prec) || opt->degree < 0 ||
        (opt->degree > 0 && (!(opt->lambda_max > 0.0) || !(opt->smoothing_range > 1.0))))
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_cg_solve: bad argument");
    hx_ctx *ctx = m->ctx;
    if (!m->cache[HX_FP64].valid || !m->cache[opt->precond_prec].valid)
        return fail(ctx, HX_ERR_NOT_READY, "hx_cg_solve: quadrature-point data missing (FP64 and preconditioner precision)");
    hx_status st = ensure_cg_ws(m);
    if (st != HX_OK) return st;
    const int pp = opt->precond_prec;
    st = ensure_cheb_ws(m, pp);
    if (st != HX_OK) return st;
    const int64_t n = 3 * m->n_nodes;
    double *dinv64 = m->w_cg + 5 * n;
    float *dinv32 = m->w_cg32 + 2 * n;
    void *dinv = pp == HX_FP64 ? (void *)dinv64 : (void *)dinv32;
    // Jacobi: inverse diagonal of the preconditioner's operator (its own precision)
    auto setup = [&]() -> hx_status {
        hx_status s2 = hx_diagonal(m, dinv, pp);
        if (s2 != HX_OK) return s2;
        HX_CUDA(ctx, hx::invert(n, dinv, dinv, pp, ctx->stream));
        return HX_OK;
    };
    auto pre = [&](const double *r, double *z, bool r32_ready) {
        return cg_precond(m, pp, opt->degree, opt->lambda_max, opt->smoothing_range, r, z, dinv, r32_ready);
    };
    st = cg_core(m, rhs, x, tol, max_iter, pp, opt->use_graph, setup, pre, iters, rel_residual);
    if (st != HX_OK) {
        const std::string e = "hx_cg_solve: " + ctx->err;
        ctx->err = e;
    }
    return st;
}

hx_status hx_measure_fma_peak(hx_ctx *ctx, int32_t prec, double *flops) {
    if (!ctx || !flops || bad_prec(prec)) return HX_ERR_ARG;
    DeviceGuard dg(ctx->device);
    HX_CUDA(ctx, dg.err);
    HX_CUDA(ctx, hx::fma_probe(prec, ctx->sm_count, flops));
    return HX_OK;
}

// ---------------------------------------------------------------------------
// batches of meshes: one persistent launch over a degree-sorted work list
// ---------------------------------------------------------------------------
}  // extern "C"

// Workspace of the batched CG (allocated by the first solve, kept for later ones)
struct BatchCg {
    int64_t total = 0, max_n = 0;
    hx::BSeg *d_seg = nullptr;
    double *w = nullptr;   // r z zold p Ap x b dinv d Kx: 10 concatenated FP64 vectors
    float *w32 = nullptr;  // r xc d Kx dinv: 5 concatenated FP32 vectors (FP32 preconditioner)
    hx::BScal *d_sc = nullptr;
    double *d_partial = nullptr, *d_dots = nullptr, *d_coef = nullptr;
    hx::BatchMesh *d_role[3] = {nullptr, nullptr, nullptr};  // p -> Ap, x -> Ap (FP64); xc -> Kx (preconditioner)
    hx::BScal *h_sc = nullptr;  // pinned
    cudaStream_t stream = nullptr;
};

struct hx_batch {
    hx_ctx *ctx = nullptr;
    std::vector<hx_mesh *> meshes;
    int law = 0;
    hx::BatchMesh *d_meshes = nullptr;
    std::vector<hx::BatchMesh> h;
    int2 *d_items[2][4] = {{nullptr, nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr, nullptr}};
    int nitems[2][4] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}};
    BatchCg cg;
};

extern "C" {

hx_status hx_batch_create(hx_ctx *ctx, hx_mesh *const *meshes, int32_t n_meshes, hx_batch **batch) {
    if (!ctx || !meshes || n_meshes < 1 || !batch) return fail(ctx, HX_ERR_ARG, "hx_batch_create: bad argument");
    *batch = nullptr;
    for (int i = 0; i < n_meshes; ++i) {
        if (!meshes[i] || meshes[i]->ctx != ctx)
            return fail(ctx, HX_ERR_ARG, "hx_batch_create: every mesh must belong to the batch's context");
        if (meshes[i]->law != meshes[0]->law) return fail(ctx, HX_ERR_ARG, "hx_batch_create: meshes of one batch share a law");
    }
    hx_batch *b = new hx_batch();
    b->ctx = ctx;
    b->meshes.assign(meshes, meshes + n_meshes);
    b->law = meshes[0]->law;
    b->h.resize(n_meshes);
    cudaError_t e = cudaMalloc((void **)&b->d_meshes, sizeof(hx::BatchMesh) * n_meshes);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(ctx, e, "hx_batch_create");
    }
    *batch = b;
    return HX_OK;
}

void hx_batch_destroy(hx_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->ctx->stream);
    if (b->cg.stream) cudaStreamSynchronize(b->cg.stream);
    dfree(b->d_meshes);
    for (auto &row : b->d_items)
        for (auto *p : row) dfree(p);
    void *cg[] = {b->cg.d_seg, b->cg.w, b->cg.w32, b->cg.d_sc, b->cg.d_partial, b->cg.d_dots, b->cg.d_coef,
                  b->cg.d_role[0], b->cg.d_role[1], b->cg.d_role[2]};
    for (void *p : cg) dfree(p);
    if (b->cg.h_sc) cudaFreeHost(b->cg.h_sc);
    if (b->cg.stream) cudaStreamDestroy(b->cg.stream);
    delete b;
}

// Work list of (mesh, tile) items of a batch, highest degree first, built once
// per (prec, storage).
static hx_status batch_items(hx_batch *b, int prec, int storage) {
    hx_ctx *ctx = b->ctx;
    if (b->nitems[prec][storage] >= 0) return HX_OK;
    const hx::BatchOps *ops = hx::batch_ops(prec);
    const int n = (int)b->meshes.size();
    std::vector<int2> items;
    for (int p = HX_PMAX; p >= HX_PMIN; --p)
        for (int i = 0; i < n; ++i) {
            const hx_mesh *m = b->meshes[i];
            if (m->p != p) continue;
            const int epb = ops->epb(p, b->law, storage);
            if (epb < 1) return fail(ctx, HX_ERR_UNSUPPORTED, "batch: degree not in the batch unit");
            const int nt = (m->n_elem + epb - 1) / epb;
            for (int t = 0; t < nt; ++t) items.push_back(make_int2(i, t));
        }
    HX_CUDA(ctx, cudaMalloc((void **)&b->d_items[prec][storage], sizeof(int2) * (items.size() + 1)));
    if (!items.empty())
        HX_CUDA(ctx, cudaMemcpy(b->d_items[prec][storage], items.data(), sizeof(int2) * items.size(),
                                cudaMemcpyHostToDevice));
    b->nitems[prec][storage] = (int)items.size();
    return HX_OK;
}

hx_status hx_batch_tangent_apply(hx_batch *b, const void *const *du_dev, void *const *out_dev, int32_t prec) {
    if (!b || !du_dev || !out_dev || bad_prec(prec)) return fail(b ? b->ctx : nullptr, HX_ERR_ARG, "hx_batch_tangent_apply: bad argument");
    hx_ctx *ctx = b->ctx;
    const int n = (int)b->meshes.size();
    const int storage = b->meshes[0]->cache[prec].storage;
    for (int i = 0; i < n; ++i) {
        const QpCache &c = b->meshes[i]->cache[prec];
        if (!c.valid) return fail(ctx, HX_ERR_NOT_READY, "hx_batch_tangent_apply: a mesh has no quadrature-point data at this precision");
        if (c.storage != storage) return fail(ctx, HX_ERR_ARG, "hx_batch_tangent_apply: meshes of a batch must share the storage strategy");
        if (!du_dev[i] || !out_dev[i] || du_dev[i] == out_dev[i]) return fail(ctx, HX_ERR_ARG, "hx_batch_tangent_apply: bad vector");
    }
    if (storage == HX_RECOMPUTE)
        return fail(ctx, HX_ERR_UNSUPPORTED, "hx_batch_tangent_apply: batches run the caching strategies");
    const hx::BatchOps *ops = hx::batch_ops(prec);
    hx_status st = batch_items(b, prec, storage);
    if (st != HX_OK) return st;
    for (int i = 0; i < n; ++i) {
        hx_mesh *m = b->meshes[i];
        b->h[i].m = view(m, prec);
        b->h[i].du = du_dev[i];
        b->h[i].out = out_dev[i];
        b->h[i].n_dofs = 3 * m->n_nodes;
    }
    // pageable source: the copy is staged before the call returns
    HX_CUDA(ctx, cudaMemcpyAsync(b->d_meshes, b->h.data(), sizeof(hx::BatchMesh) * n, cudaMemcpyHostToDevice, ctx->stream));
    HX_CUDA(ctx, ops->zero(b->d_meshes, n, ctx->stream));
    HX_CUDA(ctx, ops->apply(b->law, storage, b->d_meshes, b->d_items[prec][storage], b->nitems[prec][storage], ctx->stream));
    ctx->launches += 2;
    for (int i = 0; i < n; ++i) {
        hx_mesh *m = b->meshes[i];
        if (m->n_constrained) {
            HX_CUDA(ctx, hx::copy_idx(m->d_cidx, m->n_constrained, du_dev[i], out_dev[i], prec, ctx->stream));
            ctx->launches++;
        }
    }
    return HX_OK;
}

// ---------------------------------------------------------------------------
// batched CG: every mesh of a batch solves its own constrained system; the
// meshes iterate in lockstep so that each operator application is one
// persistent launch over all of them
// ---------------------------------------------------------------------------
// K_i v_i for every mesh in one launch, from a device array of per-mesh
// (view, du, out) entries prepared before any capture; constrained rows copied
// (sc non-null: meshes no longer active are skipped; their role entries carry
// the same flags)
static hx_status batch_apply_role(hx_batch *b, const hx::BatchMesh *role, int prec, int storage, const void *du,
                                  void *out, const hx::BScal *sc) {
    hx_ctx *ctx = b->ctx;
    const hx::BatchOps *ops = hx::batch_ops(prec);
    const int n = (int)b->meshes.size();
    HX_CUDA(ctx, ops->zero(role, n, ctx->stream));
    HX_CUDA(ctx, ops->apply(b->law, storage, role, b->d_items[prec][storage], b->nitems[prec][storage], ctx->stream));
    HX_CUDA(ctx, hx::bcopy_idx(n, b->cg.d_seg, du, out, prec, sc, ctx->stream));
    ctx->launches += 3;
    return HX_OK;
}

hx_status hx_batch_cg_solve(hx_batch *b, const double *const *rhs_dev, double *const *x_dev, double tol,
                            int32_t max_iter, int32_t degree, double smoothing_range, int32_t precond_prec,
                            int32_t use_graph, int32_t *iters, double *rel_residual) {
    if (!b || !rhs_dev || !x_dev || !(tol > 0.0) || max_iter < 0 || degree < 1 || !(smoothing_range > 1.0) ||
        bad_prec(precond_prec))
        return fail(b ? b->ctx : nullptr, HX_ERR_ARG, "hx_batch_cg_solve: bad argument");
    hx_ctx *ctx = b->ctx;
    const int nm = (int)b->meshes.size();
    const int pp = precond_prec;
    const int storage = b->meshes[0]->cache[HX_FP64].storage;
    for (int i = 0; i < nm; ++i) {
        const hx_mesh *m = b->meshes[i];
        if (!m->cache[HX_FP64].valid || !m->cache[pp].valid)
            return fail(ctx, HX_ERR_NOT_READY, "hx_batch_cg_solve: every mesh needs quadrature-point data in FP64 and in the preconditioner's precision");
        if (m->cache[HX_FP64].storage != storage || m->cache[pp].storage != storage)
            return fail(ctx, HX_ERR_ARG, "hx_batch_cg_solve: the meshes' caches must share one storage strategy");
        if (!rhs_dev[i] || !x_dev[i] || (const void *)rhs_dev[i] == (const void *)x_dev[i])
            return fail(ctx, HX_ERR_ARG, "hx_batch_cg_solve: bad vector");
    }
    if (storage == HX_RECOMPUTE) return fail(ctx, HX_ERR_UNSUPPORTED, "hx_batch_cg_solve: batches run the caching strategies");
    hx_status st = batch_items(b, HX_FP64, storage);
    if (st == HX_OK) st = batch_items(b, pp, storage);
    if (st != HX_OK) return st;

    BatchCg &w = b->cg;
    // segments (each starts on a multiple of 4 entries)
    std::vector<hx::BSeg> seg(nm);
    int64_t total = 0, max_n = 0;
    for (int i = 0; i < nm; ++i) {
        const hx_mesh *m = b->meshes[i];
        seg[i].off = total;
        seg[i].n = 3 * m->n_nodes;
        seg[i].x = x_dev[i];
        seg[i].rhs = rhs_dev[i];
        seg[i].cidx = m->d_cidx;
        seg[i].ncon = m->n_constrained;
        total += (seg[i].n + 3) / 4 * 4;
        max_n = std::max(max_n, seg[i].n);
    }
    if (w.total != total) {
        void *old[] = {w.d_seg, w.w, w.w32, w.d_sc, w.d_partial, w.d_dots, w.d_coef, w.d_role[0], w.d_role[1],
                       w.d_role[2]};
        for (void *p : old) dfree(p);
        if (w.h_sc) cudaFreeHost(w.h_sc);
        w = BatchCg{w.total, w.max_n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                    {nullptr, nullptr, nullptr}, nullptr, w.stream};
        HX_CUDA(ctx, cudaMalloc((void **)&w.d_seg, sizeof(hx::BSeg) * nm));
        HX_CUDA(ctx, cudaMalloc((void **)&w.w, 10 * (size_t)total * sizeof(double) + 64));
        HX_CUDA(ctx, cudaMalloc((void **)&w.w32, 5 * (size_t)total * sizeof(float) + 64));
        HX_CUDA(ctx, cudaMalloc((void **)&w.d_sc, sizeof(hx::BScal) * nm));
        HX_CUDA(ctx, cudaMalloc((void **)&w.d_partial, sizeof(double) * 3 * hx::BRB * nm));
        HX_CUDA(ctx, cudaMalloc((void **)&w.d_dots, sizeof(double) * 3 * nm));
        for (auto &r : w.d_role) HX_CUDA(ctx, cudaMalloc((void **)&r, sizeof(hx::BatchMesh) * nm));
        HX_CUDA(ctx, cudaHostAlloc((void **)&w.h_sc, sizeof(hx::BScal) * nm, cudaHostAllocDefault));
        w.total = total;
    }
    w.max_n = max_n;
    dfree(w.d_coef);
    w.d_coef = nullptr;
    HX_CUDA(ctx, cudaMalloc((void **)&w.d_coef, sizeof(double) * 2 * degree * nm));
    if (!w.stream) HX_CUDA(ctx, cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking));
    HX_CUDA(ctx, cudaMemcpy(w.d_seg, seg.data(), sizeof(hx::BSeg) * nm, cudaMemcpyHostToDevice));
    double *r = w.w, *z = r + total, *zold = z + total, *p = zold + total, *Ap = p + total, *xw = Ap + total,
           *bw = xw + total, *dinv = bw + total, *d64 = dinv + total, *Kx64 = d64 + total;
    float *r32 = w.w32, *xc32 = r32 + total, *d32 = xc32 + total, *Kx32 = d32 + total, *dinv32 = Kx32 + total;

    // per mesh: D^-1 (FP64, on the caller's stream), lambda_max and the Chebyshev coefficients
    std::vector<double> coef(2 * (size_t)degree * nm);
    for (int i = 0; i < nm; ++i) {
        hx_mesh *m = b->meshes[i];
        st = hx_diagonal(m, dinv + seg[i].off, HX_FP64);
        if (st != HX_OK) return st;
        HX_CUDA(ctx, hx::invert(seg[i].n, dinv + seg[i].off, dinv + seg[i].off, HX_FP64, ctx->stream));
        double lam = 0.0;
        st = hx_estimate_lambda_max(m, dinv + seg[i].off, 20, 7, &lam);
        if (st != HX_OK) return st;
        lam *= 1.2;
        const double a = lam / smoothing_range, bl = lam, theta = 0.5 * (bl + a), delta = 0.5 * (bl - a);
        double rho_prev = 0.0;
        for (int k = 0; k < degree; ++k) {
            double cd, cr, rho;
            if (k == 0) {
                rho = delta / theta;
                cd = 0.0;
                cr = 1.0 / theta;
            } else {
                rho = 1.0 / (2.0 * theta / delta - rho_prev);
                cd = rho * rho_prev;
                cr = 2.0 * rho / delta;
            }
            coef[((size_t)i * degree + k) * 2 + 0] = cd;
            coef[((size_t)i * degree + k) * 2 + 1] = cr;
            rho_prev = rho;
        }
    }
    HX_CUDA(ctx, cudaMemcpy(w.d_coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice));
    // per-mesh operator entries of the three applies
    {
        std::vector<hx::BatchMesh> role(nm);
        auto fill = [&](int k, int prec, const void *du_base, void *out_base) -> cudaError_t {
            const size_t sz = prec == HX_FP64 ? sizeof(double) : sizeof(float);
            for (int i = 0; i < nm; ++i) {
                role[i].m = view(b->meshes[i], prec);
                role[i].du = (const char *)du_base + sz * seg[i].off;
                role[i].out = (char *)out_base + sz * seg[i].off;
                role[i].n_dofs = seg[i].n;
                // the iteration's applies skip converged meshes; the residual apply (k = 1) never does
                role[i].active = k == 1 ? nullptr : &w.d_sc[i].active;
            }
            return cudaMemcpy(w.d_role[k], role.data(), sizeof(hx::BatchMesh) * nm, cudaMemcpyHostToDevice);
        };
        HX_CUDA(ctx, fill(0, HX_FP64, p, Ap));
        HX_CUDA(ctx, fill(1, HX_FP64, xw, Ap));
        if (pp == HX_FP32)
            HX_CUDA(ctx, fill(2, HX_FP32, xc32, Kx32));
        else
            HX_CUDA(ctx, fill(2, HX_FP64, z, Kx64));
    }

    // the rest runs on the batch's private stream (capturable), after the caller's work
    cudaStream_t user = ctx->stream;
    cudaEvent_t ev;
    HX_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    HX_CUDA(ctx, cudaEventRecord(ev, user));
    HX_CUDA(ctx, cudaStreamWaitEvent(w.stream, ev, 0));
    ctx->stream = w.stream;
    struct Restore {
        hx_ctx *c;
        cudaStream_t u;
        cudaEvent_t e;
        ~Restore() {
            cudaEventRecord(e, c->stream);
            cudaStreamWaitEvent(u, e, 0);
            c->stream = u;
            cudaEventDestroy(e);
        }
    } restore{ctx, user, ev};
    cudaStream_t s = ctx->stream;
    if (pp == HX_FP32) HX_CUDA(ctx, hx::to_f32(total, dinv, dinv32, s));

    // z = Chebyshev(degree)-Jacobi applied to r, per mesh, in pp (meshes no longer active skipped)
    const hx::BScal *act = w.d_sc;
    auto precond = [&]() -> hx_status {
        for (int k = 0; k < degree; ++k) {
            if (pp == HX_FP32) {
                if (k > 0) {
                    hx_status q = batch_apply_role(b, w.d_role[2], HX_FP32, storage, xc32, Kx32, act);
                    if (q != HX_OK) return q;
                }
                HX_CUDA(ctx, hx::bcheb(nm, max_n, w.d_seg, w.d_coef, degree, k, r32, k ? Kx32 : nullptr, dinv32, d32,
                                       xc32, HX_FP32, act, s));
            } else {
                if (k > 0) {
                    hx_status q = batch_apply_role(b, w.d_role[2], HX_FP64, storage, z, Kx64, act);
                    if (q != HX_OK) return q;
                }
                HX_CUDA(ctx, hx::bcheb(nm, max_n, w.d_seg, w.d_coef, degree, k, r, k ? Kx64 : nullptr, dinv, d64, z,
                                       HX_FP64, act, s));
            }
            ctx->launches++;
        }
        if (pp == HX_FP32) {
            HX_CUDA(ctx, hx::to_f64(total, xc32, z, s));
            ctx->launches++;
        }
        return HX_OK;
    };

    // every mesh active for the first preconditioner application
    for (int i = 0; i < nm; ++i) {
        w.h_sc[i] = hx::BScal{};
        w.h_sc[i].active = 1;
    }
    HX_CUDA(ctx, cudaMemcpyAsync(w.d_sc, w.h_sc, sizeof(hx::BScal) * nm, cudaMemcpyHostToDevice, s));
    // r = b - K x; z = M r; p = zold = z
    HX_CUDA(ctx, hx::bcopy(nm, max_n, w.d_seg, xw, 0, s));
    HX_CUDA(ctx, hx::bcopy(nm, max_n, w.d_seg, bw, 2, s));
    st = batch_apply_role(b, w.d_role[1], HX_FP64, storage, xw, Ap, nullptr);
    if (st != HX_OK) return st;
    HX_CUDA(ctx, hx::bsub(total, bw, Ap, r, s));
    if (pp == HX_FP32) HX_CUDA(ctx, hx::to_f32(total, r, r32, s));
    st = precond();
    if (st != HX_OK) return st;
    HX_CUDA(ctx, cudaMemcpyAsync(p, z, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
    HX_CUDA(ctx, cudaMemcpyAsync(zold, z, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
    HX_CUDA(ctx, hx::bdots(nm, w.d_seg, 3, r, z, r, r, bw, bw, w.d_partial, w.d_dots, nullptr, s));
    HX_CUDA(ctx, hx::bscal_init(nm, w.d_sc, w.d_dots, tol, s));
    ctx->launches += 8;

    auto body = [&]() -> hx_status {
        hx_status q = batch_apply_role(b, w.d_role[0], HX_FP64, storage, p, Ap, act);
        if (q != HX_OK) return q;
        HX_CUDA(ctx, hx::bdots(nm, w.d_seg, 1, p, Ap, nullptr, nullptr, nullptr, nullptr, w.d_partial, w.d_dots, act,
                               s));
        HX_CUDA(ctx, hx::bscal_alpha(nm, w.d_sc, w.d_dots, s));
        HX_CUDA(ctx, hx::bxr(nm, max_n, w.d_seg, w.d_sc, p, Ap, xw, r, pp == HX_FP32 ? r32 : nullptr, s));
        q = precond();
        if (q != HX_OK) return q;
        HX_CUDA(ctx, hx::bdots(nm, w.d_seg, 3, r, z, r, zold, r, r, w.d_partial, w.d_dots, act, s));
        HX_CUDA(ctx, hx::bscal_beta(nm, w.d_sc, w.d_dots, s));
        HX_CUDA(ctx, hx::bp(nm, max_n, w.d_seg, w.d_sc, z, p, zold, s));
        HX_CUDA(ctx, cudaMemcpyAsync(w.h_sc, w.d_sc, sizeof(hx::BScal) * nm, cudaMemcpyDeviceToHost, s));
        ctx->launches += 8;
        return HX_OK;
    };
    cudaGraphExec_t exec = nullptr;
    if (use_graph) {
        cudaGraph_t graph = nullptr;
        HX_CUDA(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        hx_status q = body();
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (q != HX_OK) {
            if (graph) cudaGraphDestroy(graph);
            return q;
        }
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaGraphInstantiate");
    }
    struct ExecGuard {
        cudaGraphExec_t e;
        ~ExecGuard() {
            if (e) cudaGraphExecDestroy(e);
        }
    } eg{exec};
    HX_CUDA(ctx, cudaMemcpyAsync(w.h_sc, w.d_sc, sizeof(hx::BScal) * nm, cudaMemcpyDeviceToHost, s));
    HX_CUDA(ctx, cudaStreamSynchronize(s));
    auto any_active = [&]() {
        for (int i = 0; i < nm; ++i)
            if (w.h_sc[i].active) return true;
        return false;
    };
    for (int it = 0; it < max_iter && any_active(); ++it) {
        if (exec) {
            HX_CUDA(ctx, cudaGraphLaunch(exec, s));
        } else {
            st = body();
            if (st != HX_OK) return st;
        }
        HX_CUDA(ctx, cudaStreamSynchronize(s));
    }
    // true residuals; the solutions back to the caller's vectors
    st = batch_apply_role(b, w.d_role[1], HX_FP64, storage, xw, Ap, nullptr);
    if (st != HX_OK) return st;
    HX_CUDA(ctx, hx::bsub(total, bw, Ap, r, s));
    HX_CUDA(ctx, hx::bdots(nm, w.d_seg, 2, r, r, bw, bw, nullptr, nullptr, w.d_partial, w.d_dots, nullptr, s));
    HX_CUDA(ctx, hx::bcopy(nm, max_n, w.d_seg, xw, 1, s));
    std::vector<double> dots(3 * (size_t)nm);
    HX_CUDA(ctx, cudaMemcpyAsync(dots.data(), w.d_dots, sizeof(double) * 3 * nm, cudaMemcpyDeviceToHost, s));
    HX_CUDA(ctx, cudaMemcpyAsync(w.h_sc, w.d_sc, sizeof(hx::BScal) * nm, cudaMemcpyDeviceToHost, s));
    HX_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->launches += 4;
    int n_bad = 0, n_open = 0;
    std::string bad_list;
    for (int i = 0; i < nm; ++i) {
        double rel = dots[3 * i + 1] > 0.0 ? std::sqrt(dots[3 * i] / dots[3 * i + 1]) : 0.0;
        if (w.h_sc[i].bad || !(rel == rel)) {
            rel = std::nan("");
            if (n_bad++ < 8) bad_list += (bad_list.empty() ? "" : ", ") + std::to_string(i);
        } else if (rel > tol) {
            ++n_open;
        }
        if (iters) iters[i] = w.h_sc[i].iters;
        if (rel_residual) rel_residual[i] = rel;
    }
    if (n_bad) return fail(ctx, HX_ERR_NAN, "hx_batch_cg_solve: CG breakdown (NaN or non-positive curvature) on " +
                                                std::to_string(n_bad) + " mesh(es): " + bad_list);
    if (n_open) return fail(ctx, HX_ERR_NOT_CONVERGED, "hx_batch_cg_solve: tolerance not reached on " +
                                                           std::to_string(n_open) + " mesh(es)");
    return HX_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// external loads and Newton's method (Alg. 1)
// ---------------------------------------------------------------------------
hx_status hx_body_force(hx_mesh *m, const double b[3], double *f_dev) {
    if (!m || !b || !f_dev) return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_body_force: bad argument");
    hx_ctx *ctx = m->ctx;
    const hx::PrecOps *ops = hx::prec_ops(m->p, HX_FP64);
    const hx::MeshView v = view(m, HX_FP64);
    HX_CUDA(ctx, cudaMemsetAsync(f_dev, 0, 3 * (size_t)m->n_nodes * sizeof(double), ctx->stream));
    HX_CUDA(ctx, ops->body_force(v, b, f_dev, ctx->stream));
    ctx->launches += 1;
    return HX_OK;
}

hx_status hx_newton_solve(hx_mesh *m, double *u, const double *f_ext, const hx_newton_options *o,
                          hx_newton_report *rep) {
    if (!m || !u || !o || !(o->eps_abs >= 0.0) || !(o->eps_rel >= 0.0) || o->max_newton < 0 ||
        o->storage < HX_RECOMPUTE || o->storage > HX_SPATIAL_TENSORS || bad_prec(o->precond_prec) ||
        o->cg_degree < 0 || !(o->cg_tol > 0.0) || o->cg_max_iter < 1 || o->lambda_iters < 1 ||
        !(o->smoothing_range > 1.0))
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_newton_solve: bad argument");
    hx_ctx *ctx = m->ctx;
    const int64_t n = 3 * m->n_nodes;
    if (!m->w_newton) HX_CUDA(ctx, cudaMalloc((void **)&m->w_newton, 3 * (size_t)n * sizeof(double) + 64));
    hx_status st = ensure_cg_ws(m);
    if (st != HX_OK) return st;
    double *r = m->w_newton, *du = r + n, *dinv = r + 2 * n;
    const int pp = o->precond_prec;
    // r = R(u) - f_ext on the free DoFs, returns ||r||_2
    auto residual_norm = [&](double *nrm) -> hx_status {
        hx_status s2 = hx_residual(m, u, r, HX_FP64);
        if (s2 != HX_OK) return s2;
        cudaStream_t s = ctx->stream;
        if (f_ext) {
            HX_CUDA(ctx, hx::axpby(n, -1.0, f_ext, 1.0, r, s));
            if (m->n_constrained) HX_CUDA(ctx, hx::set_idx(m->d_cidx, m->n_constrained, 0.0, r, HX_FP64, s));
        }
        HX_CUDA(ctx, hx::dots(n, 1, r, r, nullptr, nullptr, nullptr, nullptr, m->d_partial, m->d_dots, s));
        double h = 0.0;
        HX_CUDA(ctx, cudaMemcpyAsync(&h, m->d_dots, sizeof h, cudaMemcpyDeviceToHost, s));
        HX_CUDA(ctx, cudaStreamSynchronize(s));
        ctx->launches += 3;
        if (!(h == h)) return fail(ctx, HX_ERR_NAN, "hx_newton_solve: NaN in the residual");
        *nrm = std::sqrt(h);
        return HX_OK;
    };
    double res0 = 0.0, res = 0.0;
    st = residual_norm(&res0);
    if (st != HX_OK) return st;
    res = res0;
    int k = 0, cg_total = 0;
    hx_status lin = HX_OK;
    while (res > o->eps_abs && res > o->eps_rel * res0 && k < o->max_newton) {
        if (o->mg) {  // p-multigrid preconditioned update
            st = hx_precompute_qp(m, u, HX_FP64, o->storage);
            if (st == HX_OK) st = hx_mg_setup(o->mg, u);
            if (st != HX_OK) return st;
            HX_CUDA(ctx, hx::axpby(n, -1.0, r, 0.0, r, ctx->stream));
            HX_CUDA(ctx, cudaMemsetAsync(du, 0, n * sizeof(double), ctx->stream));
            int32_t it = 0;
            double rel = 0.0;
            lin = hx_mg_cg_solve(o->mg, r, du, o->cg_tol, o->cg_max_iter, 1, &it, &rel);
            if (lin != HX_OK && lin != HX_ERR_NOT_CONVERGED) return lin;
            cg_total += it;
            HX_CUDA(ctx, hx::axpby(n, 1.0, du, 1.0, u, ctx->stream));
            ++k;
            st = residual_norm(&res);
            if (st != HX_OK) return st;
            continue;
        }
        // update quadrature point data at u_k (both precisions the solve uses)
        st = hx_precompute_qp(m, u, HX_FP64, o->storage);
        if (st == HX_OK && pp != HX_FP64) st = hx_precompute_qp(m, u, pp, o->storage);
        if (st == HX_OK) st = hx_sync(ctx, -1);  // reports J <= 0 met at the new state
        if (st != HX_OK) return st;
        // eigenvalue bound of D^-1 K for the Chebyshev preconditioner
        double lam = 0.0;
        st = hx_diagonal(m, dinv, HX_FP64);
        if (st != HX_OK) return st;
        HX_CUDA(ctx, hx::invert(n, dinv, dinv, HX_FP64, ctx->stream));
        st = hx_estimate_lambda_max(m, dinv, o->lambda_iters, 7 + (uint64_t)k, &lam);
        if (st != HX_OK) return st;
        // K du = -r
        HX_CUDA(ctx, hx::axpby(n, -1.0, r, 0.0, r, ctx->stream));
        HX_CUDA(ctx, cudaMemsetAsync(du, 0, n * sizeof(double), ctx->stream));
        hx_cg_options cg{o->cg_degree, 1.2 * lam, o->smoothing_range, pp, 1};
        int32_t it = 0;
        double rel = 0.0;
        lin = hx_cg_solve(m, r, du, o->cg_tol, o->cg_max_iter, &cg, &it, &rel);
        if (lin != HX_OK && lin != HX_ERR_NOT_CONVERGED) return lin;  // breakdown: no usable update
        cg_total += it;
        HX_CUDA(ctx, hx::axpby(n, 1.0, du, 1.0, u, ctx->stream));
        ctx->launches += 3;
        ++k;
        st = residual_norm(&res);
        if (st != HX_OK) return st;
    }
    const bool ok = res <= o->eps_abs || res <= o->eps_rel * res0;
    if (rep) {
        rep->newton_iters = k;
        rep->cg_iters = cg_total;
        rep->res0 = res0;
        rep->res = res;
        rep->converged = ok ? 1 : 0;
    }
    if (!ok) return fail(ctx, HX_ERR_NOT_CONVERGED, "hx_newton_solve: Newton iteration limit reached");
    return HX_OK;
}

hx_status hx_material_eval(hx_mesh *m, int32_t elem, int32_t form, int32_t prec, int64_t n, const double *G,
                           const double *H, double *S, double *P, double *dP) {
    if (!m || bad_prec(prec) || form < 0 || form > 2 || n < 0 || elem < 0 || elem >= std::max(m->n_elem, 1) ||
        (n > 0 && (!G || !H || !S || !P || !dP)))
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_material_eval: bad argument");
    hx_ctx *ctx = m->ctx;
    const hx::MeshView v = view(m, prec);
    HX_CUDA(ctx, hx::prec_ops(m->p, prec)->material_eval(v, elem, form, n, G, H, S, P, dP, ctx->stream));
    ctx->launches += 1;
    return HX_OK;
}

// ---------------------------------------------------------------------------
// p-multigrid preconditioner (Sec. 6): degrees p, floor(p/2), ..., 1 on the
// same structured box, Chebyshev-Jacobi smoothing on every level, Chebyshev
// iterations on the coarsest, transfers by interpolation between the
// Lagrange spaces (prolongation) and its transpose (restriction)
// ---------------------------------------------------------------------------
struct hx_mg {
    hx_ctx *ctx = nullptr;
    std::vector<hx_mesh *> lv;  // lv[0] = the caller's mesh (not owned)
    std::vector<hx::InterpTab> down;  // lv[l] -> lv[l+1] state transfer: finer function at coarser nodes
    std::vector<hx::InterpTab> up;    // lv[l+1] -> lv[l] prolongation: coarser function at finer nodes
    std::vector<void *> b, x, t, dinv;  // per level, in the preconditioner's precision
    std::vector<double *> dinv64;       // per level, FP64 inverse diagonal (spectral estimate)
    std::vector<double *> u;  // linearization state per level (FP64), l >= 1
    std::vector<double> lam;
    std::vector<int> hpair;   // hpair[l] = 1: lv[l+1] is the 2x h-coarsening of lv[l] (degree 1)
    double *A_c = nullptr;    // coarsest level: assembled FP64 tangent (column-major), for the coarse CG
    double *I_c = nullptr;    // identity of the coarsest level's size (the assembly's unit vectors)
    int n_c = 0;
    int *d_cit = nullptr;     // iterations of the last coarse CG
    hx_mg_options opt{};
    bool ready = false;
};

static hx::InterpTab make_tab(int ps, int pd) {
    hx::InterpTab t{};
    t.ps = ps;
    t.pd = pd;
    const std::vector<double> xs = gll_points(ps), xd = gll_points(pd);
    for (int a = 0; a <= pd; ++a)
        for (int b = 0; b <= ps; ++b) {
            const double v = lagrange(xs, b, xd[a]);
            t.M[a][b] = std::fabs(v) < 1e-15 ? 0.0 : v;
        }
    return t;
}

void hx_mg_destroy(hx_mg *g) {
    if (!g) return;
    if (g->ctx) cudaStreamSynchronize(g->ctx->stream);
    for (size_t l = 0; l < g->lv.size(); ++l) {
        dfree(g->b[l]);
        dfree(g->x[l]);
        dfree(g->t[l]);
        dfree(g->dinv[l]);
        dfree(g->dinv64[l]);
        if (l > 0) {
            dfree(g->u[l]);
            hx_destroy_mesh(g->lv[l]);
        }
    }
    dfree(g->A_c);
    dfree(g->I_c);
    dfree(g->d_cit);
    delete g;
}

hx_status hx_mg_create(hx_mesh *m, const hx_mg_options *opt, hx_mg **out) {
    if (!m || !opt || !out || bad_prec(opt->precond_prec) || opt->smoother_degree < 1 || opt->coarse_degree < 1 ||
        !(opt->smoothing_range > 1.0) || !(opt->coarse_range > 1.0) || opt->lambda_iters < 1 ||
        opt->storage < HX_RECOMPUTE || opt->storage > HX_SPATIAL_TENSORS || opt->min_degree < 1 ||
        !(opt->coarse_weight > 0.0) || opt->coarse_weight > 1.0 || opt->h_levels < 0 || opt->coarse_cg_iters < 0 ||
        (opt->coarse_cg_iters > 0 && !(opt->coarse_cg_tol > 0.0)))
        return fail(m ? m->ctx : nullptr, HX_ERR_ARG, "hx_mg_create: bad argument");
    hx_ctx *ctx = m->ctx;
    if (!m->structured)
        return fail(ctx, HX_ERR_UNSUPPORTED, "hx_mg_create: levels are built for structured boxes only");
    const int nx = m->nx, ny = m->ny, nz = m->nz;
    // the constraints must be whole faces, component by component
    bool face[6][3] = {};
    const int p = m->p;
    const int64_t Nx = (int64_t)nx * p + 1, Ny = (int64_t)ny * p + 1, Nz = (int64_t)nz * p + 1;
    auto on_face = [&](int f, int64_t I, int64_t J, int64_t K, int64_t NX, int64_t NY, int64_t NZ) {
        return f == 0 ? I == 0 : f == 1 ? I == NX - 1 : f == 2 ? J == 0 : f == 3 ? J == NY - 1 : f == 4 ? K == 0 : K == NZ - 1;
    };
    const std::vector<uint8_t> &dm = m->h_dirichlet;
    if (!dm.empty()) {
        for (int f = 0; f < 6; ++f)
            for (int c = 0; c < 3; ++c) {
                bool all = true;
                for (int64_t n = 0; n < Nx * Ny * Nz && all; ++n) {
                    const int64_t I = n % Nx, J = (n / Nx) % Ny, K = n / (Nx * Ny);
                    if (on_face(f, I, J, K, Nx, Ny, Nz) && !dm[3 * n + c]) all = false;
                }
                face[f][c] = all;
            }
        for (int64_t n = 0; n < Nx * Ny * Nz; ++n) {
            const int64_t I = n % Nx, J = (n / Nx) % Ny, K = n / (Nx * Ny);
            for (int c = 0; c < 3; ++c) {
                bool want = false;
                for (int f = 0; f < 6; ++f) want = want || (face[f][c] && on_face(f, I, J, K, Nx, Ny, Nz));
                if (want != (dm[3 * n + c] != 0))
                    return fail(ctx, HX_ERR_UNSUPPORTED, "hx_mg_create: constraints must cover whole faces per component");
            }
        }
    }
    hx_mg *g = new hx_mg();
    g->ctx = ctx;
    g->opt = *opt;
    g->lv.push_back(m);
    while (g->lv.back()->p / 2 >= opt->min_degree) {
        const int pc = g->lv.back()->p / 2;
        const int64_t Mx = (int64_t)nx * pc + 1, My = (int64_t)ny * pc + 1, Mz = (int64_t)nz * pc + 1;
        std::vector<uint8_t> mask(3 * Mx * My * Mz, 0);
        bool any = false;
        for (int64_t n = 0; n < Mx * My * Mz; ++n) {
            const int64_t I = n % Mx, J = (n / Mx) % My, K = n / (Mx * My);
            for (int c = 0; c < 3; ++c)
                for (int f = 0; f < 6; ++f)
                    if (face[f][c] && on_face(f, I, J, K, Mx, My, Mz)) {
                        mask[3 * n + c] = 1;
                        any = true;
                    }
        }
        hx_mesh_desc d{};
        d.n_elem = m->n_elem;
        d.p = pc;
        d.geo_degree = m->g;
        d.n_nodes = Mx * My * Mz;
        d.geo_nodes = m->h_geo_nodes.data();
        d.n_geo_nodes = m->n_geo;
        d.geo_conn = m->h_geo_conn.data();
        d.dof_conn = nullptr;
        d.nx = nx;
        d.ny = ny;
        d.nz = nz;
        d.dirichlet = any ? mask.data() : nullptr;
        d.fibre_frames = m->h_frames.empty() ? nullptr : m->h_frames.data();
        hx_mesh *c = nullptr;
        hx_status st = hx_setup_mesh(ctx, &d, &m->h_mat, &c);
        if (st != HX_OK) {
            hx_mg_destroy(g);
            return st;
        }
        g->lv.push_back(c);
    }
    g->hpair.assign(g->lv.size(), 0);
    // h-levels: halve the degree-1 box while every direction has an even
    // number of elements; a coarse vertex is the fine lattice vertex at twice
    // its index (found through the fine element's corner), so any trilinear
    // box coarsens, nested or not
    for (int h = 0; h < opt->h_levels; ++h) {
        hx_mesh *f = g->lv.back();
        if (f->p != 1 || f->g != 1 || f->nx % 2 || f->ny % 2 || f->nz % 2) break;
        const int cx = f->nx / 2, cy = f->ny / 2, cz = f->nz / 2;
        const int64_t Vx = cx + 1, Vy = cy + 1, Vz = cz + 1;
        std::vector<double> verts(3 * Vx * Vy * Vz);
        for (int64_t n = 0; n < Vx * Vy * Vz; ++n) {
            const int64_t I = 2 * (n % Vx), J = 2 * ((n / Vx) % Vy), K = 2 * (n / (Vx * Vy));
            const int64_t ex = I < f->nx ? I : f->nx - 1, ey = J < f->ny ? J : f->ny - 1, ez = K < f->nz ? K : f->nz - 1;
            const int64_t e = ex + f->nx * (ey + (int64_t)f->ny * ez);
            const int corner = (int)(I - ex) + 2 * (int)(J - ey) + 4 * (int)(K - ez);
            const int64_t v = f->h_geo_conn[8 * e + corner];
            for (int c = 0; c < 3; ++c) verts[3 * n + c] = f->h_geo_nodes[3 * v + c];
        }
        const int64_t ne = (int64_t)cx * cy * cz;
        std::vector<int32_t> gconn(8 * ne);
        std::vector<double> frames;
        if (!f->h_frames.empty()) frames.resize(9 * ne);
        for (int64_t e = 0; e < ne; ++e) {
            const int64_t ex = e % cx, ey = (e / cx) % cy, ez = e / ((int64_t)cx * cy);
            for (int corner = 0; corner < 8; ++corner)
                gconn[8 * e + corner] = (int32_t)((ex + (corner & 1)) + Vx * ((ey + ((corner >> 1) & 1)) + Vy * (ez + (corner >> 2))));
            if (!frames.empty()) {  // the frame of the coarse element's first child
                const int64_t fe = 2 * ex + f->nx * (2 * ey + (int64_t)f->ny * 2 * ez);
                for (int k = 0; k < 9; ++k) frames[9 * e + k] = f->h_frames[9 * fe + k];
            }
        }
        std::vector<uint8_t> mask(3 * Vx * Vy * Vz, 0);
        bool any = false;
        for (int64_t n = 0; n < Vx * Vy * Vz; ++n) {
            const int64_t I = n % Vx, J = (n / Vx) % Vy, K = n / (Vx * Vy);
            for (int c = 0; c < 3; ++c)
                for (int fc = 0; fc < 6; ++fc)
                    if (face[fc][c] && on_face(fc, I, J, K, Vx, Vy, Vz)) {
                        mask[3 * n + c] = 1;
                        any = true;
                    }
        }
        hx_mesh_desc d{};
        d.n_elem = (int32_t)ne;
        d.p = 1;
        d.geo_degree = 1;
        d.n_nodes = Vx * Vy * Vz;
        d.geo_nodes = verts.data();
        d.n_geo_nodes = Vx * Vy * Vz;
        d.geo_conn = gconn.data();
        d.dof_conn = nullptr;
        d.nx = cx;
        d.ny = cy;
        d.nz = cz;
        d.dirichlet = any ? mask.data() : nullptr;
        d.fibre_frames = frames.empty() ? nullptr : frames.data();
        hx_mesh *c = nullptr;
        hx_status st = hx_setup_mesh(ctx, &d, &m->h_mat, &c);
        if (st != HX_OK) {
            hx_mg_destroy(g);
            return st;
        }
        g->hpair.back() = 1;
        g->lv.push_back(c);
        g->hpair.push_back(0);
    }
    const size_t L = g->lv.size();
    const int pp = opt->precond_prec;
    if (L > 16) {
        hx_mg_destroy(g);
        return fail(ctx, HX_ERR_UNSUPPORTED, "hx_mg_create: more than 16 levels");
    }
    if (opt->coarse_cg_iters > 0) {
        const int64_t nc = 3 * g->lv.back()->n_nodes;
        if (nc > hx::COARSE_MAX) {
            hx_mg_destroy(g);
            return fail(ctx, HX_ERR_UNSUPPORTED, "hx_mg_create: the coarsest level has " + std::to_string(nc) +
                                                     " DoFs, more than the coarse CG's " +
                                                     std::to_string(hx::COARSE_MAX));
        }
        g->n_c = (int)nc;
        std::vector<double> eye((size_t)nc * nc, 0.0);
        for (int64_t i = 0; i < nc; ++i) eye[(size_t)(i * nc + i)] = 1.0;
        cudaError_t e = cudaMalloc((void **)&g->A_c, eye.size() * sizeof(double) + 64);
        if (e == cudaSuccess) e = cudaMalloc((void **)&g->I_c, eye.size() * sizeof(double) + 64);
        if (e == cudaSuccess) e = cudaMalloc((void **)&g->d_cit, sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(g->I_c, eye.data(), eye.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            hx_mg_destroy(g);
            return cuda_fail(ctx, e, "hx_mg_create (coarse matrix)");
        }
    }
    g->b.assign(L, nullptr);
    g->x.assign(L, nullptr);
    g->t.assign(L, nullptr);
    g->dinv.assign(L, nullptr);
    g->dinv64.assign(L, nullptr);
    g->u.assign(L, nullptr);
    g->lam.assign(L, 0.0);
    for (size_t l = 0; l < L; ++l) {
        const size_t n = 3 * (size_t)g->lv[l]->n_nodes;
        const size_t bytes = n * prec_size(pp) + 64;
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = cudaMalloc(&g->b[l], bytes);
        if (e == cudaSuccess) e = cudaMalloc(&g->x[l], bytes);
        if (e == cudaSuccess) e = cudaMalloc(&g->t[l], bytes);
        if (e == cudaSuccess) e = cudaMalloc(&g->dinv[l], bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&g->dinv64[l], n * sizeof(double) + 64);
        if (e == cudaSuccess && l > 0) e = cudaMalloc((void **)&g->u[l], n * sizeof(double) + 64);
        if (e != cudaSuccess) {
            hx_mg_destroy(g);
            return cuda_fail(ctx, e, "hx_mg_create");
        }
        if (l + 1 < L) {  // (unused for an h-pair: both levels have degree 1)
            g->down.push_back(make_tab(g->lv[l]->p, g->lv[l + 1]->p));
            g->up.push_back(make_tab(g->lv[l + 1]->p, g->lv[l]->p));
        }
    }
    *out = g;
    return HX_OK;
}

hx_status hx_mg_info(const hx_mg *g, int32_t *n_levels, int32_t *degrees) {
    if (!g || !n_levels) return HX_ERR_ARG;
    *n_levels = (int32_t)g->lv.size();
    if (degrees)
        for (size_t l = 0; l < g->lv.size(); ++l) degrees[l] = g->lv[l]->p;
    return HX_OK;
}

hx_status hx_mg_level(const hx_mg *g, int32_t level, int32_t *p, int32_t *nx, int32_t *ny, int32_t *nz) {
    if (!g || level < 0 || level >= (int32_t)g->lv.size() || !p || !nx || !ny || !nz) return HX_ERR_ARG;
    const hx_mesh *lm = g->lv[level];
    *p = lm->p;
    *nx = lm->nx;
    *ny = lm->ny;
    *nz = lm->nz;
    return HX_OK;
}

hx_status hx_mg_coarse_iters(const hx_mg *g, int32_t *iters) {
    if (!g || !iters) return HX_ERR_ARG;
    *iters = -1;
    if (!g->d_cit) return HX_OK;
    int v = -1;
    HX_CUDA(g->ctx, cudaStreamSynchronize(g->ctx->stream));
    HX_CUDA(g->ctx, cudaMemcpy(&v, g->d_cit, sizeof v, cudaMemcpyDeviceToHost));
    *iters = v;
    return HX_OK;
}

hx_status hx_mg_setup(hx_mg *g, const double *u_dev) {
    if (!g || !u_dev) return fail(g ? g->ctx : nullptr, HX_ERR_ARG, "hx_mg_setup: bad argument");
    hx_ctx *ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    const int pp = g->opt.precond_prec;
    const size_t L = g->lv.size();
    g->ready = false;
    for (size_t l = 0; l < L; ++l) {
        hx_mesh *lm = g->lv[l];
        const double *ul = u_dev;
        if (l > 0) {
            // linearization point of the coarser level: the finer state at its nodes
            const double *uf = l == 1 ? u_dev : g->u[l - 1];
            if (g->hpair[l - 1])
                HX_CUDA(ctx, hx::h_inject(lm->nx, lm->ny, lm->nz, uf, g->u[l], s));
            else
                HX_CUDA(ctx, hx::interp(g->down[l - 1], lm->nx, lm->ny, lm->nz, uf, g->u[l], 0, HX_FP64, s));
            ul = g->u[l];
            ctx->launches += 1;
        }
        hx_status st = hx_precompute_qp(lm, ul, HX_FP64, g->opt.storage);
        if (st == HX_OK && pp != HX_FP64) st = hx_precompute_qp(lm, ul, pp, g->opt.storage);
        if (st != HX_OK) return st;
        // Jacobi and the spectral bound of D^-1 K (FP64), then D^-1 in the
        // smoother's precision
        double *d64 = g->dinv64[l];
        st = hx_diagonal(lm, d64, HX_FP64);
        if (st != HX_OK) return st;
        const int64_t n = 3 * lm->n_nodes;
        HX_CUDA(ctx, hx::invert(n, d64, d64, HX_FP64, s));
        st = hx_estimate_lambda_max(lm, d64, g->opt.lambda_iters, 11 + l, &g->lam[l]);
        if (st != HX_OK) return st;
        g->lam[l] *= 1.2;
        if (pp == HX_FP32)
            HX_CUDA(ctx, hx::to_f32(n, d64, (float *)g->dinv[l], s));
        else
            HX_CUDA(ctx, cudaMemcpyAsync(g->dinv[l], d64, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        st = ensure_cheb_ws(lm, pp);
        if (st != HX_OK) return st;
    }
    if (g->n_c > 0) {  // the coarse CG's matrix: the coarsest tangent (FP64) applied to unit vectors
        hx_mesh *cm = g->lv.back();
        for (int j = 0; j < g->n_c; ++j) {
            hx_status st = apply_dev(cm, g->I_c + (size_t)j * g->n_c, g->A_c + (size_t)j * g->n_c, HX_FP64);
            if (st != HX_OK) return st;
        }
    }
    {
        hx_status st = hx_sync(ctx, -1);  // J <= 0 met at a level's state
        if (st != HX_OK) return st;
    }
    g->ready = true;
    return HX_OK;
}

// one V-cycle on level l: x = V(b) (zero start), all vectors in pp precision
static hx_status vcycle(hx_mg *g, size_t l, const void *b, void *x) {
    hx_ctx *ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    const int pp = g->opt.precond_prec;
    hx_mesh *lm = g->lv[l];
    const int64_t n = 3 * lm->n_nodes;
    if (l + 1 == g->lv.size()) {
        if (g->n_c > 0) {  // FP64 Jacobi-CG on the assembled coarsest tangent
            HX_CUDA(ctx, hx::coarse_pcg(g->n_c, g->A_c, g->dinv64[l], b, x, g->opt.coarse_cg_iters, g->opt.coarse_cg_tol,
                                        g->d_cit, pp, s));
            ctx->launches++;
            return HX_OK;
        }
        return cheb_run(lm, b, x, g->dinv[l], g->opt.coarse_degree, g->lam[l], g->opt.coarse_range, 1, pp);
    }
    hx_status st = cheb_run(lm, b, x, g->dinv[l], g->opt.smoother_degree, g->lam[l], g->opt.smoothing_range, 1, pp);
    if (st != HX_OK) return st;
    // t = b - K x, restricted to the coarser level
    st = apply_dev(lm, x, g->t[l], pp);
    if (st != HX_OK) return st;
    HX_CUDA(ctx, hx::axpby_p(n, 1.0, b, -1.0, g->t[l], pp, s));
    hx_mesh *cm = g->lv[l + 1];
    const int64_t nc = 3 * cm->n_nodes;
    if (g->hpair[l]) {
        HX_CUDA(ctx, hx::h_restrict(cm->nx, cm->ny, cm->nz, g->t[l], g->b[l + 1], pp, s));
    } else {
        HX_CUDA(ctx, cudaMemsetAsync(g->b[l + 1], 0, nc * prec_size(pp), s));
        HX_CUDA(ctx, hx::interp_t(g->up[l], lm->nx, lm->ny, lm->nz, g->t[l], g->b[l + 1], pp, s));
    }
    if (cm->n_constrained) HX_CUDA(ctx, hx::set_idx(cm->d_cidx, cm->n_constrained, 0.0, g->b[l + 1], pp, s));
    st = vcycle(g, l + 1, g->b[l + 1], g->x[l + 1]);
    if (st != HX_OK) return st;
    if (g->opt.coarse_weight != 1.0)
        HX_CUDA(ctx, hx::axpby_p(3 * cm->n_nodes, g->opt.coarse_weight, g->x[l + 1], 0.0, g->x[l + 1], pp, s));
    if (g->hpair[l])
        HX_CUDA(ctx, hx::h_prolong(cm->nx, cm->ny, cm->nz, g->x[l + 1], x, 1, pp, s));
    else
        HX_CUDA(ctx, hx::interp(g->up[l], lm->nx, lm->ny, lm->nz, g->x[l + 1], x, 1, pp, s));
    if (lm->n_constrained) HX_CUDA(ctx, hx::set_idx(lm->d_cidx, lm->n_constrained, 0.0, x, pp, s));
    ctx->launches += 5;
    return cheb_run(lm, b, x, g->dinv[l], g->opt.smoother_degree, g->lam[l], g->opt.smoothing_range, 0, pp);
}

hx_status hx_mg_vcycle(hx_mg *g, const void *b_dev, void *x_dev) {
    if (!g || !b_dev || !x_dev) return fail(g ? g->ctx : nullptr, HX_ERR_ARG, "hx_mg_vcycle: bad argument");
    if (!g->ready) return fail(g->ctx, HX_ERR_NOT_READY, "hx_mg_vcycle: call hx_mg_setup first");
    return vcycle(g, 0, b_dev, x_dev);
}

hx_status hx_mg_transfer(hx_mg *g, int32_t level, int32_t dir, const void *src_dev, void *dst_dev, int32_t prec) {
    if (!g || level < 0 || level + 1 >= (int32_t)g->lv.size() || dir < 0 || dir > 2 || bad_prec(prec) || !src_dev ||
        !dst_dev)
        return fail(g ? g->ctx : nullptr, HX_ERR_ARG, "hx_mg_transfer: bad argument");
    hx_ctx *ctx = g->ctx;
    hx_mesh *fm = g->lv[level];
    cudaStream_t s = ctx->stream;
    hx_mesh *cmh = g->lv[level + 1];
    if (g->hpair[level]) {
        if (dir == 0)
            HX_CUDA(ctx, hx::h_prolong(cmh->nx, cmh->ny, cmh->nz, src_dev, dst_dev, 0, prec, s));
        else if (dir == 1)
            HX_CUDA(ctx, hx::h_restrict(cmh->nx, cmh->ny, cmh->nz, src_dev, dst_dev, prec, s));
        else if (prec == HX_FP64)
            HX_CUDA(ctx, hx::h_inject(cmh->nx, cmh->ny, cmh->nz, (const double *)src_dev, (double *)dst_dev, s));
        else
            return fail(ctx, HX_ERR_ARG, "hx_mg_transfer: the state transfer is FP64");
    } else if (dir == 0) {  // prolongation: level+1 -> level
        HX_CUDA(ctx, hx::interp(g->up[level], fm->nx, fm->ny, fm->nz, src_dev, dst_dev, 0, prec, s));
    } else if (dir == 1) {  // restriction (transpose): level -> level+1
        HX_CUDA(ctx, cudaMemsetAsync(dst_dev, 0, 3 * (size_t)g->lv[level + 1]->n_nodes * prec_size(prec), s));
        HX_CUDA(ctx, hx::interp_t(g->up[level], fm->nx, fm->ny, fm->nz, src_dev, dst_dev, prec, s));
    } else {  // state transfer: level -> level+1
        HX_CUDA(ctx, hx::interp(g->down[level], fm->nx, fm->ny, fm->nz, src_dev, dst_dev, 0, prec, s));
    }
    ctx->launches += 1;
    return HX_OK;
}

hx_status hx_mg_cg_solve(hx_mg *g, const double *rhs, double *x, double tol, int32_t max_iter, int32_t use_graph,
                         int32_t *iters, double *rel_residual) {
    if (!g || !rhs || !x || max_iter < 0 || !(tol > 0.0))
        return fail(g ? g->ctx : nullptr, HX_ERR_ARG, "hx_mg_cg_solve: bad argument");
    hx_ctx *ctx = g->ctx;
    if (!g->ready) return fail(ctx, HX_ERR_NOT_READY, "hx_mg_cg_solve: call hx_mg_setup first");
    hx_mesh *m = g->lv[0];
    const int pp = g->opt.precond_prec;
    hx_status st = ensure_cg_ws(m);
    if (st != HX_OK) return st;
    const int64_t n = 3 * m->n_nodes;
    auto setup = []() -> hx_status { return HX_OK; };
    auto pre = [&](const double *r, double *z, bool r32_ready) -> hx_status {
        cudaStream_t s = ctx->stream;
        if (pp == HX_FP32) {
            float *r32 = m->w_cg32, *z32 = m->w_cg32 + n;
            if (!r32_ready) HX_CUDA(ctx, hx::to_f32(n, r, r32, s));
            hx_status s2 = vcycle(g, 0, r32, z32);
            if (s2 != HX_OK) return s2;
            HX_CUDA(ctx, hx::to_f64(n, z32, z, s));
            ctx->launches += 2;
            return HX_OK;
        }
        return vcycle(g, 0, r, z);
    };
    st = cg_core(m, rhs, x, tol, max_iter, pp, use_graph, setup, pre, iters, rel_residual);
    if (st != HX_OK) ctx->err = "hx_mg_cg_solve: " + ctx->err;
    return st;
}
