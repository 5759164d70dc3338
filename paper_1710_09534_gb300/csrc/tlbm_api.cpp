// C ABI of the lattice library (declared in include/tlbm.h): argument
// validation, derived parameters (Eqs. 7, 9, 12, 18a, 38), geometry
// classification and the compacted near-wall list, workspace carving, and the
// per-step launches on the caller's stream.
#include "tlbm.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "tlbm_internal.h"
#include "tlbm_ops.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int ok()
{
    g_err.clear();
    return TLB_OK;
}

#define TLB_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(TLB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));           \
    } while (0)

constexpr int64_t kAlign = 256;
constexpr int kMassParts = 608;  // 4 x 152 SMs
constexpr int kMaxDrops = 256;   // contact-line results kept per call

int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }


// precision argument: TLB_FP64 .. TLB_BF16, optionally | TLB_INPLACE
bool precision_ok(int precision)
{
    const int base = precision & ~TLB_INPLACE;
    return base >= TLB_FP64 && base <= TLB_BF16;
}

// Rows of set-up input one pass of the in-place tlb_set_fields stages in the
// order-parameter planes: c1, c2 with 3 halo rows on each side, ux, uy, p.
int band_rows(int64_t stage_doubles, int nx) { return (int)((stage_doubles / nx - 12) / 5); }

tlb::Layout layout_for(int nx, int ny, int precision_flags)
{
    tlb::Layout L;
    const int precision = precision_flags & ~TLB_INPLACE;
    L.inplace = (precision_flags & TLB_INPLACE) != 0;
    L.pitch = (int)align_up(nx, 32);
    L.plane = (int64_t)L.pitch * ny;
    const int64_t es = (int64_t)tlb::elem_for(precision);
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        const int64_t at = off;
        off = align_up(off + bytes, kAlign);
        return at;
    };
    const int nd = tlb::ndist_for(precision);
    L.fA = take(nd * L.plane * es);
    L.fB = L.inplace ? L.fA : take(nd * L.plane * es);
    L.cu = take(4 * L.plane * (int64_t)tlb::cu_elem_for(precision));
    if (L.inplace) {
        // c_1, c_2 planes of the arithmetic type; at least one staged set-up row
        const int64_t relem = precision == TLB_FP64 ? 8 : 4;
        L.cpl_bytes = std::max<int64_t>(2 * L.plane * relem, 17 * (int64_t)nx * 8);
        L.cpl = take(L.cpl_bytes);
    }
    L.cls = take(L.plane);
    L.list = take((int64_t)nx * ny * 4);
    L.part = take((int64_t)kMassParts * 4 * 8);
    L.diag = take(4 * 8);
    // contact-line scratch: wall-row c and column heights (2 nx doubles),
    // up to kMaxDrops results (4 doubles each) and the drop count
    L.contact = take((2 * (int64_t)nx + 4 * kMaxDrops) * 8 + 16);
    L.total = off;
    return L;
}

}  // namespace


namespace {

// Site classification with the same semantics as the device site_of().
int host_site(const tlb_lattice* L, int x, int y, int64_t* idx)
{
    if (x < 0 || x >= L->nx) {
        const int e = L->edge[x < 0 ? 0 : 1];
        if (e != TLB_EDGE_PERIODIC) return e == TLB_EDGE_WETTING ? tlb::ST_WET : tlb::ST_NEUTRAL;
        x = x < 0 ? x + L->nx : x - L->nx;
    }
    if (y < 0 || y >= L->ny) {
        const int e = L->edge[y < 0 ? 2 : 3];
        if (e == TLB_EDGE_LID) return tlb::ST_VOID;
        if (e != TLB_EDGE_PERIODIC) return e == TLB_EDGE_WETTING ? tlb::ST_WET : tlb::ST_NEUTRAL;
        y = y < 0 ? y + L->ny : y - L->ny;
    }
    const int64_t i = (int64_t)y * L->nx + x;
    if (idx) *idx = i;
    if (L->mask[i] == TLB_NODE_WETTING_SOLID) return tlb::ST_WET;
    if (L->mask[i] == TLB_NODE_NEUTRAL_SOLID) return tlb::ST_NEUTRAL;
    if (L->edge[3] == TLB_EDGE_LID && y == L->ny - 1) return tlb::ST_LID;
    return tlb::ST_FLUID;
}

// Node classes and the near-wall list from the host mask; uploads both.
int build_geometry(tlb_lattice* L)
{
    const int nx = L->nx, ny = L->ny, pitch = L->lay.pitch;
    L->cls.assign((size_t)L->lay.plane, (uint8_t)tlb::ST_NEUTRAL);
    std::vector<uint32_t> list;
    list.reserve((size_t)nx * 4);
    for (int y = 0; y < ny; y++) {
        for (int x = 0; x < nx; x++) {
            const int kind = host_site(L, x, y, nullptr);
            uint8_t c = (uint8_t)kind;
            if (kind == tlb::ST_FLUID) {
                bool interior = true;
                for (int dy = -2; dy <= 2 && interior; dy++)
                    for (int dx = -2; dx <= 2 && interior; dx++)
                        if (host_site(L, x + dx, y + dy, nullptr) != tlb::ST_FLUID) interior = false;
                if (interior) c |= tlb::CLS_INTERIOR;
            }
            L->cls[(size_t)y * pitch + x] = c;
            if ((kind == tlb::ST_FLUID || kind == tlb::ST_LID) && !(c & tlb::CLS_INTERIOR))
                list.push_back(((uint32_t)y << 16) | (uint32_t)x);
        }
    }
    L->nlist = (int64_t)list.size();
    L->hlist = list;
    TLB_CUDA(cudaMemcpyAsync(L->ws + L->lay.cls, L->cls.data(), L->cls.size(), cudaMemcpyHostToDevice,
                             L->stream));
    if (!list.empty())
        TLB_CUDA(cudaMemcpyAsync(L->ws + L->lay.list, list.data(), list.size() * 4, cudaMemcpyHostToDevice,
                                 L->stream));
    TLB_CUDA(cudaStreamSynchronize(L->stream));
    return TLB_OK;
}

constexpr int kProfSlots = 512;

// Fold the recorded events (per step: interior start/end, near-wall
// start/end) into the per-kernel totals (synchronizes).
int prof_fold(tlb_lattice* L)
{
    if (L->ev_used == 0) return TLB_OK;
    TLB_CUDA(cudaEventSynchronize(L->ev[4 * (L->ev_used - 1) + 1]));
    TLB_CUDA(cudaEventSynchronize(L->ev[4 * (L->ev_used - 1) + 3]));
    for (int i = 0; i < L->ev_used; i++) {
        float a = 0, b = 0;
        TLB_CUDA(cudaEventElapsedTime(&a, L->ev[4 * i], L->ev[4 * i + 1]));
        TLB_CUDA(cudaEventElapsedTime(&b, L->ev[4 * i + 2], L->ev[4 * i + 3]));
        L->prof_ms[0] += a;
        L->prof_ms[1] += b;
        L->prof_n[0] += 1;
        L->prof_n[1] += L->nlist > 0 ? 1 : 0;
    }
    L->ev_used = 0;
    return TLB_OK;
}

// One step's launches: `interior` on the lattice's stream and `wall` on the
// side stream between a fork after `pre` (work both depend on) and a join,
// then `post` on the lattice's stream; with profiling, events around both.
template <typename Pre, typename Interior, typename Wall, typename Post>
int step_launches(tlb_lattice* L, Pre pre, Interior interior, Wall wall, Post post)
{
    int rc;
    cudaEvent_t* ev = nullptr;
    if (L->prof) {
        if (L->ev_used == kProfSlots && (rc = prof_fold(L))) return rc;
        ev = &L->ev[4 * L->ev_used];
        TLB_CUDA(cudaEventRecord(ev[0], L->stream));
    }
    TLB_CUDA(pre());
    const bool two = L->nlist > 0;
    // the near-wall launch goes first, so that its few blocks are resident
    // before the interior grid takes the SMs
    if (two) {
        TLB_CUDA(cudaEventRecord(L->fork, L->stream));
        TLB_CUDA(cudaStreamWaitEvent(L->side, L->fork, 0));
        if (ev) TLB_CUDA(cudaEventRecord(ev[2], L->side));
        TLB_CUDA(wall(L->side));
        if (ev) TLB_CUDA(cudaEventRecord(ev[3], L->side));
        TLB_CUDA(cudaEventRecord(L->join, L->side));
    }
    TLB_CUDA(interior());
    if (ev) TLB_CUDA(cudaEventRecord(ev[1], L->stream));
    if (two) {
        TLB_CUDA(cudaStreamWaitEvent(L->stream, L->join, 0));
    } else if (ev) {
        TLB_CUDA(cudaEventRecord(ev[2], L->stream));
        TLB_CUDA(cudaEventRecord(ev[3], L->stream));
    }
    TLB_CUDA(post());
    if (ev) L->ev_used++;
    return TLB_OK;
}

int check_handle(tlb_lattice* L)
{
    if (!L) return fail(TLB_EINVAL, "null lattice handle");
    TLB_CUDA(cudaSetDevice(L->device));
    // a member of a batch: let queued batch steps finish before touching it
    return tlb::batch_sync(L->batch);
}

bool finite_all(const tlb_params* p)
{
    const double* v = (const double*)p;
    for (size_t i = 0; i < sizeof(tlb_params) / sizeof(double); i++)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

extern "C" {

int64_t tlb_workspace_bytes(int nx, int ny, int precision)
{
    if (nx < 3 || ny < 3 || nx > 32768 || ny > 32768) return fail(TLB_EINVAL, "lattice size %dx%d out of range", nx, ny);
    if (!precision_ok(precision)) return fail(TLB_EINVAL, "unknown precision %d", precision);
    ok();
    return layout_for(nx, ny, precision).total;
}

int tlb_create_lattice(int nx, int ny, int precision, const int32_t edges[4], void* dev_workspace,
                       int64_t ws_bytes, void* cuda_stream, tlb_lattice** out)
{
    if (!out) return fail(TLB_EINVAL, "out is null");
    *out = nullptr;
    if (nx < 3 || ny < 3 || nx > 32768 || ny > 32768) return fail(TLB_EINVAL, "lattice size %dx%d out of range", nx, ny);
    if (!precision_ok(precision)) return fail(TLB_EINVAL, "unknown precision %d", precision);
    if (!edges) return fail(TLB_EINVAL, "edges is null");
    for (int e = 0; e < 4; e++)
        if (edges[e] < TLB_EDGE_PERIODIC || edges[e] > TLB_EDGE_LID) return fail(TLB_EINVAL, "edge %d: bad kind %d", e, edges[e]);
    if ((edges[0] == TLB_EDGE_PERIODIC) != (edges[1] == TLB_EDGE_PERIODIC))
        return fail(TLB_EINVAL, "left/right edges: periodic must be paired");
    if ((edges[2] == TLB_EDGE_PERIODIC) != (edges[3] == TLB_EDGE_PERIODIC))
        return fail(TLB_EINVAL, "bottom/top edges: periodic must be paired");
    if (edges[0] == TLB_EDGE_LID || edges[1] == TLB_EDGE_LID || edges[2] == TLB_EDGE_LID)
        return fail(TLB_EINVAL, "a velocity lid is supported on the top edge only");
    if (edges[3] == TLB_EDGE_LID && ny < 6) return fail(TLB_EINVAL, "a lid needs ny >= 6");
    const tlb::Layout lay = layout_for(nx, ny, precision);
    if (!dev_workspace) return fail(TLB_EINVAL, "workspace is null");
    if (((uintptr_t)dev_workspace) % kAlign) return fail(TLB_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < lay.total)
        return fail(TLB_ENOMEM, "workspace has %lld bytes, needs %lld", (long long)ws_bytes, (long long)lay.total);
    auto* L = new tlb_lattice;
    L->nx = nx;
    L->ny = ny;
    L->precision = precision & ~TLB_INPLACE;
    for (int e = 0; e < 4; e++) L->edge[e] = edges[e];
    L->stream = (cudaStream_t)cuda_stream;
    L->ws = (char*)dev_workspace;
    L->lay = lay;
    L->ops = &tlb::ops_for(L->precision, false);
    L->geo.nx = nx;
    L->geo.ny = ny;
    L->geo.pitch = lay.pitch;
    L->geo.plane = lay.plane;
    for (int e = 0; e < 4; e++) L->geo.edge[e] = edges[e];
    L->mask.assign((size_t)nx * ny, 0);
    cudaError_t e = cudaGetDevice(&L->device);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L->side, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (L->done) cudaEventDestroy(L->done);
        if (L->fork) cudaEventDestroy(L->fork);
        if (L->join) cudaEventDestroy(L->join);
        delete L;
        return fail(TLB_ECUDA, "device set-up failed: %s", cudaGetErrorString(e));
    }
    int rc = build_geometry(L);
    if (rc == TLB_OK) {
        cudaError_t z = cudaMemsetAsync(L->ws + lay.fA, 0, (size_t)(lay.cls - lay.fA), L->stream);
        if (z == cudaSuccess) z = cudaStreamSynchronize(L->stream);
        if (z != cudaSuccess) rc = fail(TLB_ECUDA, "workspace clear failed: %s", cudaGetErrorString(z));
    }
    if (rc != TLB_OK) {
        cudaEventDestroy(L->done);
        cudaEventDestroy(L->fork);
        cudaEventDestroy(L->join);
        cudaStreamDestroy(L->side);
        delete L;
        return rc;
    }
    *out = L;
    return ok();
}

int tlb_set_geometry(tlb_lattice* L, const uint8_t* host_mask)
{
    int rc = check_handle(L);
    if (rc) return rc;
    std::vector<uint8_t> m((size_t)L->n(), 0);
    if (host_mask) {
        for (int64_t i = 0; i < L->n(); i++) {
            if (host_mask[i] > TLB_NODE_NEUTRAL_SOLID) return fail(TLB_EINVAL, "mask value %d at node %lld", host_mask[i], (long long)i);
            m[i] = host_mask[i];
        }
    }
    if (L->edge[3] == TLB_EDGE_LID) {
        for (int y = L->ny - 2; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++)
                if (m[(size_t)y * L->nx + x]) return fail(TLB_EINVAL, "with a lid, rows ny-2 and ny-1 must be fluid");
    }
    L->mask.swap(m);
    rc = build_geometry(L);
    if (rc) return rc;
    tlb::batch_member_changed(L->batch);
    L->have_fields = false;
    return ok();
}

int tlb_set_params(tlb_lattice* L, const tlb_params* p)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (!p) return fail(TLB_EINVAL, "params is null");
    if (!finite_all(p)) return fail(TLB_EINVAL, "non-finite parameter");
    if (p->sigma12 <= 0 || p->sigma13 <= 0 || p->sigma23 <= 0) return fail(TLB_EINVAL, "surface tensions must be > 0");
    const double l1 = p->sigma12 + p->sigma13 - p->sigma23;
    const double l2 = p->sigma12 + p->sigma23 - p->sigma13;
    const double l3 = p->sigma13 + p->sigma23 - p->sigma12;
    if (l1 <= 0 || l2 <= 0 || l3 < 0) return fail(TLB_EINVAL, "Eq. 7 gives lambda = (%g, %g, %g): need l1, l2 > 0, l3 >= 0", l1, l2, l3);
    if (p->D <= 0) return fail(TLB_EINVAL, "D must be > 0");
    if (p->rho1 <= 0 || p->rho2 <= 0 || p->rho3 <= 0) return fail(TLB_EINVAL, "densities must be > 0");
    if (p->nu1 <= 0 || p->nu2 <= 0 || p->nu3 <= 0) return fail(TLB_EINVAL, "viscosities must be > 0");
    if (p->tau1 <= 0.5 || p->tau2 <= 0.5) return fail(TLB_EINVAL, "tau_i must be > 1/2");
    if (p->M0 <= 0) return fail(TLB_EINVAL, "M0 must be > 0");
    if (p->collision != 0.0 && p->collision != 1.0) return fail(TLB_EINVAL, "collision must be 0 (BGK) or 1 (MRT)");
    const bool mrt = p->collision == 1.0;
    if (mrt && !(p->mrt_s_f > 0 && p->mrt_s_f < 2 && p->mrt_s_g > 0 && p->mrt_s_g < 2))
        return fail(TLB_EINVAL, "MRT rates must lie in (0, 2)");
    const double deg = 3.14159265358979323846 / 180.0;
    const double c12 = std::cos(p->theta12_deg * deg), c13 = std::cos(p->theta13_deg * deg),
                 c23 = std::cos(p->theta23_deg * deg);
    const double smax = std::fmax(p->sigma12, std::fmax(p->sigma13, p->sigma23));
    const double resid = p->sigma12 * c12 - p->sigma13 * c13 + p->sigma23 * c23;
    if (std::fabs(resid) > 1e-6 * smax)
        return fail(TLB_EINVAL, "contact angles violate Eq. 39 (residual %g)", resid);
    const double den = l1 * l2 + l1 * l3 + l2 * l3;
    const double lT = den != 0 ? 3.0 * l1 * l2 * l3 / den : 0.0;
    tlb::Prm<double>& P = L->prm;
    P.lam[0] = l1;
    P.lam[1] = l2;
    P.lam[2] = l3;
    P.lamT = lT;
    P.two_lamT = 2.0 * lT;
    P.k12D = 12.0 / p->D;
    P.k34D = 0.75 * p->D;
    P.k4D = 4.0 / p->D;
    const double tau[2] = {p->tau1, p->tau2};
    const double M[2] = {p->M0 / l1, p->M0 / l2};
    const double w[2] = {1.0 / 9.0, 1.0 / 36.0};
    for (int i = 0; i < 2; i++) {
        P.k34Dlam[i] = 0.75 * p->D * P.lam[i];
        P.eta[i] = M[i] / ((1.0 / 3.0) * (tau[i] - 0.5));
        P.inv_tau[i] = 1.0 / tau[i];
        P.omt[i] = 1.0 - 1.0 / tau[i];
        P.src_f[i] = 3.0 * (1.0 - 0.5 / tau[i]);
        P.e0[i] = (4.0 / 9.0 - 1.0) * P.eta[i] / tau[i];
        for (int c = 0; c < 2; c++) {
            P.aw[i][c] = P.eta[i] * w[c] / tau[i];
            P.bw[i][c] = 3.0 * w[c] / tau[i];
            P.sw[i][c] = P.src_f[i] * w[c];
        }
    }
    P.rho[0] = p->rho1;
    P.rho[1] = p->rho2;
    P.rho[2] = p->rho3;
    P.nu[0] = p->nu1;
    P.nu[1] = p->nu2;
    P.nu[2] = p->nu3;
    P.drho[0] = p->rho1 - p->rho3;
    P.drho[1] = p->rho2 - p->rho3;
    P.dnu[0] = p->nu1 - p->nu3;
    P.dnu[1] = p->nu2 - p->nu3;
    P.aM[0] = (p->rho1 - p->rho3) * M[0];
    P.aM[1] = (p->rho2 - p->rho3) * M[1];
    P.l3_l1 = l3 / l1;
    P.l3_l2 = l3 / l2;
    P.cos12 = c12;
    P.cos13 = c13;
    P.cos23 = c23;
    P.gx = p->gx;
    P.gy = p->gy;
    P.lid_u = p->lid_u;
    // equal densities and viscosities: constants of the uniform-property update
    P.uni = (p->rho1 == p->rho3 && p->rho2 == p->rho3 && p->nu1 == p->nu3 && p->nu2 == p->nu3) ? 1.0 : 0.0;
    {
        const double itg = 1.0 / (3.0 * p->nu3 + 0.5);
        P.inv_rho3 = 1.0 / p->rho3;
        P.inv_taug3 = itg;
        P.omtg3 = 1.0 - itg;
        P.kG3 = 1.0 - 0.5 * itg;
        for (int c = 0; c < 2; c++) {
            P.Rw3[c] = w[c] * p->rho3 * itg;
            P.Kw3[c] = w[c] * P.kG3;
        }
        P.p3tg3 = 3.0 * itg;
        P.rg3x = p->rho3 * p->gx;
        P.rg3y = p->rho3 * p->gy;
    }
    // constants of the scaled stencils: grad9s = 12 grad, lap9s = 6 lap
    for (int i = 0; i < 2; i++) {
        P.Kl[i] = P.k12D * P.lam[i];
        P.K34l6[i] = P.k34Dlam[i] / 6.0;
        P.drho12[i] = P.drho[i] / 12.0;
        P.aM6[i] = P.aM[i] / 6.0;
        P.k3tau[i] = 3.0 / tau[i];
        P.kq[i] = 3.0 / 36.0 / tau[i];
        P.ks[i] = P.src_f[i] / 36.0;
        P.K3w3[i] = 3.0 * P.Kw3[i];
    }
    P.Kt = P.k12D * P.two_lamT;
    // mu_1 - mu_3 = (1 + l3/l1) mu_1 + (l3/l2) mu_2, mu_2 - mu_3 = (l3/l1) mu_1 + (1 + l3/l2) mu_2
    P.qa[0][0] = (1.0 + P.l3_l1) / 12.0;
    P.qa[0][1] = P.l3_l2 / 12.0;
    P.qa[1][0] = P.l3_l1 / 12.0;
    P.qa[1][1] = (1.0 + P.l3_l2) / 12.0;
    P.mrt = mrt ? 1.0 : 0.0;
    P.mrt_s_f = mrt ? p->mrt_s_f : 1.0;
    P.mrt_s_g = mrt ? p->mrt_s_g : 1.0;
    L->ops = &tlb::ops_for(L->precision, mrt);
    L->have_params = true;
    L->have_fields = false;
    tlb::batch_member_changed(L->batch);
    g_err.clear();
    if (l1 <= 0.5 * lT || l2 <= 0.5 * lT || l3 <= 0.5 * lT)
        g_err = "warning: some lambda_i <= lambda_T / 2 (outside the well-posed range of the bulk free energy)";
    return TLB_OK;
}

static int set_fields_impl(tlb_lattice* L, const double* c1, const double* c2, const double* ux,
                           const double* uy, const double* p)
{
    TLB_CUDA(L->ops->init(L->bufA(), L->cu(), L->dcls(), c1, c2, ux, uy, p, L->geo, L->prm, L->stream));
    L->have_fields = true;
    return TLB_OK;
}

// In-place lattices have no spare buffer: the host inputs go through the
// order-parameter planes in bands of rows (c1, c2 with the 3 halo rows the
// set-up window needs on each side, wrapped on a periodic y axis; ux, uy, p
// of the band itself), one set-up launch per band.
static int set_fields_banded(tlb_lattice* L, const double* c1, const double* c2, const double* ux,
                             const double* uy, const double* p)
{
    const int nx = L->nx, ny = L->ny;
    const int64_t stage_doubles = L->lay.cpl_bytes / 8;
    const int b = std::min(ny, band_rows(stage_doubles, nx));
    if (b < 1) return fail(TLB_ECUDA, "order-parameter planes too small to stage a row");
    double* st = (double*)L->cpl();
    const size_t row = (size_t)nx * 8;
    const bool wrap = L->edge[2] == TLB_EDGE_PERIODIC;
    for (int y0 = 0; y0 < ny; y0 += b) {
        const int y1 = std::min(ny, y0 + b), rows = (y1 - y0) + 6, y_b = y0 - 3;
        double* sc1 = st;
        double* sc2 = st + (size_t)rows * nx;
        double* su = sc2 + (size_t)rows * nx;
        double* sv = su + (size_t)(y1 - y0) * nx;
        double* sp = sv + (size_t)(y1 - y0) * nx;
        // runs of band rows that are consecutive lattice rows (a wrap splits them)
        for (int r = 0; r < rows;) {
            int y = y_b + r, n = rows - r;
            if (y < 0) {
                n = std::min(n, -y);
                y += ny;
            } else if (y >= ny) {
                y -= ny;
            } else {
                n = std::min(n, ny - y);
            }
            n = std::min(n, ny - y);
            if (wrap || (y_b + r >= 0 && y_b + r < ny)) {  // rows beyond a wall or lid edge are never read
                TLB_CUDA(cudaMemcpyAsync(sc1 + (size_t)r * nx, c1 + (size_t)y * nx, (size_t)n * row,
                                         cudaMemcpyHostToDevice, L->stream));
                TLB_CUDA(cudaMemcpyAsync(sc2 + (size_t)r * nx, c2 + (size_t)y * nx, (size_t)n * row,
                                         cudaMemcpyHostToDevice, L->stream));
            }
            r += n;
        }
        const size_t band = (size_t)(y1 - y0) * row;
        TLB_CUDA(cudaMemcpyAsync(su, ux + (size_t)y0 * nx, band, cudaMemcpyHostToDevice, L->stream));
        TLB_CUDA(cudaMemcpyAsync(sv, uy + (size_t)y0 * nx, band, cudaMemcpyHostToDevice, L->stream));
        if (p) TLB_CUDA(cudaMemcpyAsync(sp, p + (size_t)y0 * nx, band, cudaMemcpyHostToDevice, L->stream));
        TLB_CUDA(L->ops->init_rows(L->bufA(), L->cu(), L->dcls(), sc1, sc2, su, sv, p ? sp : nullptr, L->geo, L->prm,
                                   y0, y1, y_b, rows, L->stream));
    }
    L->have_fields = true;
    return TLB_OK;
}

int tlb_set_fields(tlb_lattice* L, const double* c1, const double* c2, const double* ux, const double* uy,
                   const double* p)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (!L->have_params) return fail(TLB_ESTATE, "set_params first");
    if (!c1 || !c2 || !ux || !uy) return fail(TLB_EINVAL, "c1, c2, ux, uy are required");
    if (L->lay.inplace) {
        rc = set_fields_banded(L, c1, c2, ux, uy, p);
        if (rc) return rc;
        TLB_CUDA(cudaStreamSynchronize(L->stream));
        return ok();
    }
    // stage the inputs in the spare distribution buffer, build the state,
    // then clear the spare buffer (solid nodes and lid slots must read zero)
    const size_t N = (size_t)L->n();
    double* stage = (double*)L->bufB();
    const double* src[5] = {c1, c2, ux, uy, p};
    for (int q = 0; q < 5; q++)
        if (src[q]) TLB_CUDA(cudaMemcpyAsync(stage + q * N, src[q], N * 8, cudaMemcpyHostToDevice, L->stream));
    rc = set_fields_impl(L, stage, stage + N, stage + 2 * N, stage + 3 * N, p ? stage + 4 * N : nullptr);
    if (rc) return rc;
    TLB_CUDA(cudaMemsetAsync(L->bufB(), 0, (size_t)(L->ops->ndist * L->lay.plane * L->ops->elem), L->stream));
    TLB_CUDA(cudaStreamSynchronize(L->stream));
    return ok();
}

int tlb_set_fields_device(tlb_lattice* L, const double* c1, const double* c2, const double* ux,
                          const double* uy, const double* p)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (!L->have_params) return fail(TLB_ESTATE, "set_params first");
    if (!c1 || !c2 || !ux || !uy) return fail(TLB_EINVAL, "c1, c2, ux, uy are required");
    rc = set_fields_impl(L, c1, c2, ux, uy, p);
    if (rc) return rc;
    if (!L->lay.inplace)
        TLB_CUDA(cudaMemsetAsync(L->bufB(), 0, (size_t)(L->ops->ndist * L->lay.plane * L->ops->elem), L->stream));
    return ok();
}

// In-place lattices: steps in even/odd pairs (an odd step leaves the usual
// layout), a last even step followed by the in-place streaming swap.
static int step_inplace(tlb_lattice* L, int64_t n)
{
    int rc;
    const bool lid = L->edge[3] == TLB_EDGE_LID;
    for (int64_t s = 0; s < n; s++) {
        const int odd = (int)(s & 1);
        rc = step_launches(
            L, [&] { return L->ops->csum_ip(L->bufA(), L->cpl(), L->dcls(), L->geo, odd, L->stream); },
            [&] { return L->ops->interior_ip(L->bufA(), L->cu(), L->cpl(), L->dcls(), L->geo, L->prm, odd, L->stream); },
            [&](cudaStream_t ws) {
                cudaError_t e = cudaSuccess;
                if (lid)
                    e = L->ops->wall_ip(L->bufA(), L->cu(), L->cpl(), L->dcls(), L->dlist(), (int)L->nlist, L->geo,
                                        L->prm, odd, 1, ws);
                if (e == cudaSuccess)
                    e = L->ops->wall_ip(L->bufA(), L->cu(), L->cpl(), L->dcls(), L->dlist(), (int)L->nlist, L->geo,
                                        L->prm, odd, 0, ws);
                return e;
            },
            [&] {
                return (!odd && s == n - 1) ? L->ops->swap_ip(L->bufA(), L->dcls(), L->geo, L->stream) : cudaSuccess;
            });
        if (rc) return rc;
    }
    return ok();
}

int tlb_step(tlb_lattice* L, int64_t n)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (n < 0) return fail(TLB_EINVAL, "negative step count");
    if (!L->have_params || !L->have_fields) return fail(TLB_ESTATE, "set_params and set_fields before step");
    if (L->batch) return fail(TLB_ESTATE, "lattice belongs to a batch: step the batch");
    if (L->lay.inplace) return step_inplace(L, n);
    for (int64_t s = 0; s < n; s++) {
        rc = step_launches(
            L, [] { return cudaSuccess; },
            [&] { return L->ops->interior(L->bufA(), L->bufB(), L->cu(), L->dcls(), L->geo, L->prm, L->stream); },
            [&](cudaStream_t ws) {
                return L->ops->wall(L->bufA(), L->bufB(), L->cu(), L->dcls(), L->dlist(), (int)L->nlist, L->geo,
                                    L->prm, ws);
            },
            [] { return cudaSuccess; });
        if (rc) return rc;
        L->cur ^= 1;
    }
    return ok();
}

int tlb_sync(tlb_lattice* L, int64_t timeout_ms)
{
    int rc = check_handle(L);
    if (rc) return rc;
    TLB_CUDA(cudaEventRecord(L->done, L->stream));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(L->done);
        if (e == cudaSuccess) return ok();
        if (e != cudaErrorNotReady) return fail(TLB_ECUDA, "stream error: %s", cudaGetErrorString(e));
        if (timeout_ms >= 0) {
            const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
            if (ms >= timeout_ms) return fail(TLB_ETIMEOUT, "work still pending after %lld ms", (long long)timeout_ms);
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int tlb_read_fields_device(tlb_lattice* L, uint32_t mask, double* dev_out)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (!L->have_params || !L->have_fields) return fail(TLB_ESTATE, "no state yet");
    if (!dev_out || (mask & ~(uint32_t)TLB_F_ALL) || !mask) return fail(TLB_EINVAL, "bad output or field mask");
    TLB_CUDA(L->ops->read(L->bufA(), L->dcls(), dev_out, mask, L->geo, L->prm, L->stream));
    return ok();
}

int tlb_read_fields(tlb_lattice* L, uint32_t mask, double* host_out)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (!L->have_params || !L->have_fields) return fail(TLB_ESTATE, "no state yet");
    if (!host_out || (mask & ~(uint32_t)TLB_F_ALL) || !mask) return fail(TLB_EINVAL, "bad output or field mask");
    // stage in the spare distribution buffer, as many FP64 planes per pass as
    // it holds (8 or more: it has >= 66 bytes per node in every precision);
    // in-place lattices stage in the order-parameter planes (1 or 2 per pass)
    const size_t N = (size_t)L->n();
    const size_t spare = L->lay.inplace ? (size_t)L->lay.cpl_bytes
                                        : (size_t)(L->ops->ndist * L->lay.plane * L->ops->elem);
    const int per_pass = (int)std::min<size_t>(10, spare / (N * 8));
    double* stage = (double*)(L->lay.inplace ? L->cpl() : L->bufB());
    size_t done = 0;
    for (int q = 0; q < 10;) {
        uint32_t sub = 0;
        int cnt = 0;
        for (; q < 10 && cnt < per_pass; q++)
            if (mask & (1u << q)) {
                sub |= 1u << q;
                cnt++;
            }
        if (!sub) continue;
        TLB_CUDA(L->ops->read(L->bufA(), L->dcls(), stage, sub, L->geo, L->prm, L->stream));
        TLB_CUDA(cudaMemcpyAsync(host_out + done * N, stage, (size_t)cnt * N * 8, cudaMemcpyDeviceToHost, L->stream));
        done += (size_t)cnt;
    }
    if (!L->lay.inplace) TLB_CUDA(cudaMemsetAsync(L->bufB(), 0, spare, L->stream));
    TLB_CUDA(cudaStreamSynchronize(L->stream));
    return ok();
}

int tlb_diagnostics(tlb_lattice* L, tlb_diag* out)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (!out) return fail(TLB_EINVAL, "out is null");
    if (!L->have_params || !L->have_fields) return fail(TLB_ESTATE, "no state yet");
    double* part = (double*)(L->ws + L->lay.part);
    double* dout = (double*)(L->ws + L->lay.diag);
    TLB_CUDA(L->ops->mass(L->bufA(), L->dcls(), part, kMassParts, dout, L->geo, L->stream));
    double h[4];
    TLB_CUDA(cudaMemcpyAsync(h, dout, sizeof h, cudaMemcpyDeviceToHost, L->stream));
    TLB_CUDA(cudaStreamSynchronize(L->stream));
    out->mass[0] = h[0];
    out->mass[1] = h[1];
    out->mass[2] = h[2];
    out->nonfinite = (int64_t)h[3];
    if (out->nonfinite > 0) return fail(TLB_EUNSTABLE, "%lld fluid nodes hold non-finite values", (long long)out->nonfinite);
    return ok();
}

int tlb_contact_angles(tlb_lattice* L, int component, double* host_out, int max_drops, int* n_drops)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (component != 1 && component != 2) return fail(TLB_EINVAL, "component must be 1 or 2");
    if (!host_out || !n_drops || max_drops < 0) return fail(TLB_EINVAL, "bad output arguments");
    if (!L->have_params || !L->have_fields) return fail(TLB_ESTATE, "no state yet");
    double* wallc = (double*)(L->ws + L->lay.contact);
    double* colh = wallc + L->nx;
    double* res = colh + L->nx;
    int* cnt = (int*)(res + 4 * kMaxDrops);
    const int keep = max_drops < kMaxDrops ? max_drops : kMaxDrops;
    TLB_CUDA(L->ops->contact(L->bufA(), L->dcls(), component, wallc, colh, res, kMaxDrops, cnt, L->geo, L->stream));
    int n = 0;
    TLB_CUDA(cudaMemcpyAsync(&n, cnt, sizeof n, cudaMemcpyDeviceToHost, L->stream));
    TLB_CUDA(cudaStreamSynchronize(L->stream));
    const int copy = n < keep ? n : keep;
    if (copy > 0) {
        TLB_CUDA(cudaMemcpyAsync(host_out, res, (size_t)copy * 4 * 8, cudaMemcpyDeviceToHost, L->stream));
        TLB_CUDA(cudaStreamSynchronize(L->stream));
    }
    *n_drops = n;
    return ok();
}

int tlb_film_thickness(tlb_lattice* L, int x, int y_top, int comps, double* h_out)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (!h_out) return fail(TLB_EINVAL, "h_out is null");
    if (x < 0 || x >= L->nx || y_top < -1 || y_top > L->ny - 2)
        return fail(TLB_EINVAL, "column %d / solid row %d outside the lattice", x, y_top);
    if (comps < 1 || comps > 3) return fail(TLB_EINVAL, "comps must be 1, 2 or 3");
    if (!L->have_params || !L->have_fields) return fail(TLB_ESTATE, "no state yet");
    double* res = (double*)(L->ws + L->lay.contact) + 2 * (size_t)L->nx;
    TLB_CUDA(L->ops->film(L->bufA(), L->dcls(), x, y_top, comps, res, L->geo, L->stream));
    TLB_CUDA(cudaMemcpyAsync(h_out, res, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    TLB_CUDA(cudaStreamSynchronize(L->stream));
    return ok();
}

// IEEE 754 binary16 and bfloat16 bit patterns to double (host side of the
// 16-bit storage formats).
static double half_bits(uint16_t h)
{
    const int e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = std::ldexp((double)m, -24);  // subnormal: m 2^-24
    else if (e == 31) v = m ? std::nan("") : INFINITY;
    else v = std::ldexp((double)(1024 + m), e - 25);  // (1 + m/1024) 2^(e-15)
    return (h & 0x8000) ? -v : v;
}
static double bf16_bits(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

int tlb_read_state(tlb_lattice* L, double* host_out)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (!host_out) return fail(TLB_EINVAL, "out is null");
    const size_t es = L->ops->elem, ces = L->ops->cu_elem, PL = (size_t)L->lay.plane, nd = (size_t)L->ops->ndist;
    const size_t dbytes = nd * PL * es;
    std::vector<char> raw(dbytes + 4 * PL * ces);
    TLB_CUDA(cudaMemcpyAsync(raw.data(), L->bufA(), dbytes, cudaMemcpyDeviceToHost, L->stream));
    TLB_CUDA(cudaMemcpyAsync(raw.data() + dbytes, L->cu(), 4 * PL * ces, cudaMemcpyDeviceToHost, L->stream));
    TLB_CUDA(cudaStreamSynchronize(L->stream));
    auto f32 = [&](size_t byte) {
        float f;
        memcpy(&f, raw.data() + byte, 4);
        return (double)f;
    };
    auto f64 = [&](size_t byte) {
        double v;
        memcpy(&v, raw.data() + byte, 8);
        return v;
    };
    const double inv16 = std::ldexp(1.0, -tlb::kF16ScaleExp);
    // population q (0..26) of pitched node i, rest populations as hi + lo
    auto pop = [&](size_t q, size_t i) {
        const bool rest = q == 0 || q == 9;
        const size_t r = q == 9 ? 1 : 0;
        if (es == 8) return f64((q * PL + i) * 8);
        if (es == 4) return rest ? f32((q * PL + i) * 4) + f32(((27 + r) * PL + i) * 4) : f32((q * PL + i) * 4);
        const size_t fr = 25 * PL * 2;  // FP32 region after the 16-bit planes
        if (rest) return f32(fr + (r * PL + i) * 4) + f32(fr + ((2 + r) * PL + i) * 4);
        // f^1_k, f^2_k share 32-bit word k-1 of a node (low, high half); g_k follow
        const size_t e = q < 9 ? (q - 1) * 2 * PL + 2 * i : (q < 18 ? (q - 10) * 2 * PL + 2 * i + 1 : (16 + (q - 18)) * PL + i);
        uint16_t b;
        memcpy(&b, raw.data() + e * 2, 2);
        return L->precision == TLB_FP16 ? half_bits(b) * inv16 : bf16_bits(b);
    };
    auto cuv = [&](size_t q, size_t i) { return ces == 8 ? f64(dbytes + (q * PL + i) * 8) : f32(dbytes + (q * PL + i) * 4); };
    const size_t N = (size_t)L->n();
    for (int q = 0; q < 31; q++) {
        // output plane q: 27 distributions, then the 4 c_i u planes
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++) {
                const size_t i = (size_t)y * L->lay.pitch + x;
                host_out[q * N + (size_t)y * L->nx + x] = q < 27 ? pop((size_t)q, i) : cuv((size_t)(q - 27), i);
            }
    }
    return ok();
}

int64_t tlb_state_bytes(tlb_lattice* L)
{
    if (!L) return fail(TLB_EINVAL, "null lattice handle");
    return L->lay.plane * ((int64_t)L->ops->ndist * (int64_t)L->ops->elem + 4 * (int64_t)L->ops->cu_elem);
}

int tlb_export_state(tlb_lattice* L, void* host_buf, int64_t bytes)
{
    int rc = check_handle(L);
    if (rc) return rc;
    const int64_t need = tlb_state_bytes(L);
    if (!host_buf || bytes < need) return fail(TLB_EINVAL, "buffer needs %lld bytes", (long long)need);
    const size_t a = (size_t)L->ops->ndist * L->lay.plane * L->ops->elem;
    TLB_CUDA(cudaMemcpyAsync(host_buf, L->bufA(), a, cudaMemcpyDeviceToHost, L->stream));
    TLB_CUDA(cudaMemcpyAsync((char*)host_buf + a, L->cu(), (size_t)need - a, cudaMemcpyDeviceToHost, L->stream));
    TLB_CUDA(cudaStreamSynchronize(L->stream));
    return ok();
}

int tlb_import_state(tlb_lattice* L, const void* host_buf, int64_t bytes)
{
    int rc = check_handle(L);
    if (rc) return rc;
    const int64_t need = tlb_state_bytes(L);
    if (!host_buf || bytes != need) return fail(TLB_EINVAL, "state must be exactly %lld bytes", (long long)need);
    if (!L->have_params) return fail(TLB_ESTATE, "set_params first");
    const size_t a = (size_t)L->ops->ndist * L->lay.plane * L->ops->elem;
    TLB_CUDA(cudaMemcpyAsync(L->bufA(), host_buf, a, cudaMemcpyHostToDevice, L->stream));
    TLB_CUDA(cudaMemcpyAsync(L->cu(), (const char*)host_buf + a, (size_t)need - a, cudaMemcpyHostToDevice, L->stream));
    if (!L->lay.inplace) TLB_CUDA(cudaMemsetAsync(L->bufB(), 0, a, L->stream));
    TLB_CUDA(cudaStreamSynchronize(L->stream));
    L->have_fields = true;
    return ok();
}

int tlb_theta12_from(double s12, double s13, double s23, double th13, double th23, double* th12)
{
    if (!th12 || s12 <= 0) return fail(TLB_EINVAL, "bad arguments");
    const double deg = 3.14159265358979323846 / 180.0;
    const double c = (s13 * std::cos(th13 * deg) - s23 * std::cos(th23 * deg)) / s12;
    if (!(std::fabs(c) <= 1.0)) return fail(TLB_EINVAL, "no theta_12 satisfies Eq. 39 (cos = %g)", c);
    *th12 = std::acos(c) / deg;
    return ok();
}

int64_t tlb_wall_nodes(tlb_lattice* L)
{
    if (!L) return fail(TLB_EINVAL, "null lattice handle");
    return L->nlist;
}

int tlb_profile(tlb_lattice* L, int enable)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (enable && L->ev.empty()) {
        L->ev.resize(4 * kProfSlots);
        for (auto& e : L->ev) TLB_CUDA(cudaEventCreate(&e));
    }
    if (!enable && (rc = prof_fold(L))) return rc;
    L->prof = enable != 0;
    L->prof_ms[0] = L->prof_ms[1] = 0;
    L->prof_n[0] = L->prof_n[1] = 0;
    L->ev_used = 0;
    return ok();
}

int tlb_profile_read(tlb_lattice* L, double ms[2], int64_t launches[2])
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (!ms || !launches) return fail(TLB_EINVAL, "null output");
    if ((rc = prof_fold(L))) return rc;
    for (int i = 0; i < 2; i++) {
        ms[i] = L->prof_ms[i];
        launches[i] = L->prof_n[i];
    }
    return ok();
}

void tlb_destroy(tlb_lattice* L)
{
    if (!L) return;
    if (L->batch) tlb_batch_remove(L->batch, L);
    for (auto e : L->ev) cudaEventDestroy(e);
    if (L->done) cudaEventDestroy(L->done);
    if (L->fork) cudaEventDestroy(L->fork);
    if (L->join) cudaEventDestroy(L->join);
    if (L->side) cudaStreamDestroy(L->side);
    delete L;
}

const char* tlb_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace tlb {

int lattice_view(tlb_lattice* L, LatticeView* v)
{
    int rc = check_handle(L);
    if (rc) return rc;
    if (!v) return fail(TLB_EINVAL, "null view");
    if (!L->have_params || !L->have_fields) return fail(TLB_ESTATE, "no state yet");
    v->dist = L->bufA();
    v->cls = L->dcls();
    v->geo = L->geo;
    v->precision = L->precision;
    v->ops = L->ops;
    v->device = L->device;
    v->stream = L->stream;
    return TLB_OK;
}

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

int clear_error() { return ok(); }

}  // namespace tlb
