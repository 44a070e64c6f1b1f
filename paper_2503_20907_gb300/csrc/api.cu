// C ABI of the spline x-ray projector (declared in include/spline_project.h):
// argument checks, the cached per-device workspace and the order of the
// kernels of one call (line setup, footprint tables, projection).
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

thread_local std::string g_err;

sp_status fail(sp_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

sp_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(SP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

constexpr int kMaxDevices = 64;

struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};

std::mutex g_mu;
Workspace g_ws[kMaxDevices];

// Workspace of at least `bytes` on the current device.
sp_status workspace(size_t bytes, void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SP_EUNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace &ws = g_ws[dev];
    if (ws.bytes < bytes) {
        if (ws.ptr) {
            // earlier calls may still use it
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            cudaFree(ws.ptr);
            ws.ptr = nullptr;
            ws.bytes = 0;
        }
        size_t grow = bytes + bytes / 4 + (1u << 20);
        e = cudaMalloc(&ws.ptr, grow);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ws.ptr = nullptr;
            return fail(SP_ENOMEM, std::string("workspace allocation failed: ") + cudaGetErrorString(e));
        }
        ws.bytes = grow;
    }
    *out = ws.ptr;
    return SP_OK;
}

bool finite(float v) { return std::isfinite(v); }

sp_status check_grid(const sp_grid *g, spx::GridDev *out)
{
    if (!g) return fail(SP_EINVAL, "grid is NULL");
    if (g->nx < 1 || g->ny < 1 || g->nx > 16384 || g->ny > 16384)
        return fail(SP_EINVAL, "grid size must be in [1, 16384]");
    if (g->degree < 0 || g->degree > 3) return fail(SP_EINVAL, "degree must be 0..3");
    if (g->basis != SP_BASIS_BSPLINE && g->basis != SP_BASIS_BOX3) return fail(SP_EINVAL, "unknown grid.basis");
    if (g->basis == SP_BASIS_BOX3 && g->degree != 1)
        return fail(SP_EINVAL, "the 3-direction box-spline needs grid.degree = 1");
    if (!finite(g->h) || !(g->h > 0.f)) return fail(SP_EINVAL, "grid spacing h must be finite and > 0");
    if (!finite(g->cx) || !finite(g->cy)) return fail(SP_EINVAL, "grid centre must be finite");
    *out = spx::GridDev{g->nx, g->ny, g->degree, g->basis, g->basis == SP_BASIS_BOX3 ? 2 : g->degree,
                        g->h, g->cx, g->cy};
    return SP_OK;
}

int64_t count_lines(const sp_lines *L)
{
    if (!L || L->reserved != 0) return -1;
    switch (L->kind) {
    case SP_LINES_THETA_Y:
    case SP_LINES_POINTS:
        return L->m >= 0 ? L->m : -1;
    case SP_LINES_PARALLEL:
    case SP_LINES_FAN: {
        if (L->n_view < 1 || L->n_det < 1) return -1;
        int64_t m = (int64_t)L->n_view * (int64_t)L->n_det;
        if (L->m != 0 && L->m != m) return -1;
        return m;
    }
    default:
        return -1;
    }
}

sp_status check_lines(const sp_lines *L, spx::LinesDev *out)
{
    if (!L) return fail(SP_EINVAL, "lines is NULL");
    if (L->reserved != 0) return fail(SP_EINVAL, "lines.reserved must be 0");
    int64_t m = count_lines(L);
    if (m < 0) return fail(SP_EINVAL, "invalid line list (kind, counts or m)");
    if (m > 0x7fffffffLL) return fail(SP_EUNSUPPORTED, "more than 2^31-1 lines");
    switch (L->kind) {
    case SP_LINES_THETA_Y:
        if (m > 0 && (!L->theta || !L->y)) return fail(SP_EINVAL, "theta/y pointers are NULL");
        break;
    case SP_LINES_POINTS:
        if (m > 0 && (!L->src || !L->dst)) return fail(SP_EINVAL, "src/dst pointers are NULL");
        break;
    case SP_LINES_PARALLEL:
        if (!L->view) return fail(SP_EINVAL, "view angles pointer is NULL");
        if (!finite(L->det0) || !finite(L->ddet)) return fail(SP_EINVAL, "det0/ddet must be finite");
        break;
    case SP_LINES_FAN:
        if (!L->view) return fail(SP_EINVAL, "view angles pointer is NULL");
        if (!finite(L->det0) || !finite(L->ddet)) return fail(SP_EINVAL, "det0/ddet must be finite");
        if (!finite(L->dso) || !finite(L->dod) || !(L->dso > 0.f) || !((double)L->dso + L->dod > 0.0))
            return fail(SP_EINVAL, "fan needs dso > 0 and dso + dod > 0");
        break;
    }
    *out = spx::LinesDev{L->kind, L->n_view, L->n_det, m, L->theta, L->y, L->src, L->dst, L->view,
                         L->det0, L->ddet, L->dso, L->dod};
    return SP_OK;
}

int64_t table_count(const spx::LinesDev &L)
{
    return L.kind == SP_LINES_PARALLEL ? (int64_t)L.n_view : L.m;
}

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Line records and footprint tables for (grid, lines) in the workspace.
// Scratch of the strip kernels: transposed coefficients, the slow-row
// counter, then (free line lists) the chunk order and its sort's scratch.
size_t order_bytes(const spx::LinesDev &L) { return spx::strip_needs_order(L) ? align_up(spx::line_order_bytes(L.m)) : 0; }

size_t extra_bytes(const spx::GridDev &g, const spx::LinesDev &L)
{
    if (!spx::strip_supported(g, L)) return 0;
    return align_up(spx::strip_scratch_bytes(g)) + 256 + order_bytes(L) +
           sizeof(unsigned) * (size_t)(2 + spx::strip_chunk_count(L));
}

int *slow_counter(const spx::GridDev &g, void *extra)
{
    return reinterpret_cast<int *>(static_cast<char *>(extra) + align_up(spx::strip_scratch_bytes(g)));
}

// The adjoint's list of chunks deferred to float strips (after the order).
unsigned *defer_area(const spx::GridDev &g, const spx::LinesDev &L, void *extra)
{
    return reinterpret_cast<unsigned *>(static_cast<char *>(extra) + align_up(spx::strip_scratch_bytes(g)) + 256 +
                                        order_bytes(L));
}

// Where the chunk order of a free line list lives (NULL for other kinds).
void *order_area(const spx::GridDev &g, const spx::LinesDev &L, void *extra)
{
    if (!extra || !spx::strip_needs_order(L) || !spx::strip_supported(g, L)) return nullptr;
    return static_cast<char *>(extra) + align_up(spx::strip_scratch_bytes(g)) + 256;
}

// Kernel paths: strip kernels (structured geometries, any degree) or the
// general warp-per-line kernels.  kPathAuto takes the strip kernels for degree
// >= 1 (at degree 0 a row has at most two candidates, too few to repay the
// row records and their sort; the strip kernels run it when asked).
// kPathGather (adjoint only): the pixel-driven gather where it applies.
enum KernelPath { kPathAuto = 0, kPathStrip = 1, kPathGeneral = 2, kPathGather = 3 };

bool use_strip(const spx::GridDev &g, const spx::LinesDev &L, void *extra, int path)
{
    return extra && spx::strip_supported(g, L) && (path == kPathStrip || (path == kPathAuto && g.kdeg >= 1));
}

// Forward projection (rec: the plan's row records, or NULL).
cudaError_t run_fwd(const spx::GridDev &g, const spx::LinesDev &L, const spx::LineHdr *hdr, const float *tabs,
                    void *extra, const float *coef, float *sino, cudaStream_t s, int path = kPathAuto,
                    const spx::StripRec *rec = nullptr)
{
    if (use_strip(g, L, extra, path))
        return spx::launch_fwd_strip(g, L, hdr, tabs, coef, extra, sino, slow_counter(g, extra), s, rec);
    return spx::launch_fwd(g, hdr, tabs, L.m, coef, sino, s);
}

// Adjoint (coef_out overwritten).
cudaError_t run_adj(const spx::GridDev &g, const spx::LinesDev &L, const spx::LineHdr *hdr, const float *tabs,
                    void *extra, const float *sino, float *coef_out, cudaStream_t s, int path = kPathAuto,
                    const spx::StripRec *rec = nullptr)
{
    if (path == kPathGather && spx::gather_supported(g, L))
        return spx::launch_adj_gather(g, L, hdr, tabs, sino, coef_out, s);
    if (use_strip(g, L, extra, path))
        return spx::launch_adj_strip(g, L, hdr, tabs, sino, extra, coef_out, slow_counter(g, extra), s, rec,
                                     defer_area(g, L, extra));
    return spx::launch_adj(g, hdr, tabs, L.m, sino, coef_out, s);
}

// Row records a plan keeps: strip-path geometries of degree >= 1 (where the
// strip kernels are the automatic choice), if they fit in a quarter of the
// device's free memory and kRecMaxBytes.
constexpr size_t kRecMaxBytes = size_t(16) << 30;

size_t rec_bytes_wanted(const spx::GridDev &g, const spx::LinesDev &L)
{
    if (!spx::strip_supported(g, L) || g.kdeg < 1 || L.m == 0) return 0;
    return (size_t)L.m * (size_t)spx::strip_rec_line_bytes(g);
}

sp_status prepare(const spx::GridDev &g, spx::LinesDev &L, cudaStream_t s,
                  spx::LineHdr **hdr, float **tabs, void **extra = nullptr)
{
    const int64_t nt = table_count(L);
    size_t hb = align_up(sizeof(spx::LineHdr) * (size_t)L.m);
    size_t tb = align_up(sizeof(float) * (size_t)spx::kTabFloats * (size_t)nt);
    size_t xb = align_up(extra_bytes(g, L));
    void *ws = nullptr;
    sp_status st = workspace(hb + tb + xb + 256, &ws);
    if (st != SP_OK) return st;
    *hdr = reinterpret_cast<spx::LineHdr *>(ws);
    *tabs = reinterpret_cast<float *>(static_cast<char *>(ws) + hb);
    if (extra) *extra = xb ? static_cast<char *>(ws) + hb + tb : nullptr;
    cudaError_t e = spx::launch_prepare(g, L, *hdr, *tabs, nt, s);
    if (e != cudaSuccess) return cuda_fail(e, "line setup and footprint tables");
    // free line lists: the chunk order of the strip kernels
    void *oa = extra ? order_area(g, L, *extra) : nullptr;
    if (oa) {
        e = spx::launch_line_order(g, L, *hdr, oa, s);
        if (e != cudaSuccess) return cuda_fail(e, "line order");
        L.order = static_cast<const int *>(oa);
    }
    return SP_OK;
}

}  // namespace

namespace spx {
// For other translation units of the library: the same argument checks and
// the same thread-local last-error message as the entry points above.
sp_status check_grid_for(const sp_grid *g, GridDev *out) { return check_grid(g, out); }
sp_status check_lines_for(const sp_lines *L, LinesDev *out) { return check_lines(L, out); }
sp_status record_error(sp_status st, const std::string &msg) { return fail(st, msg); }
sp_status record_error(sp_status st, const char *msg) { return fail(st, std::string(msg)); }
void clear_error() { g_err.clear(); }
}  // namespace spx

extern "C" {

int64_t sp_lines_count(const sp_lines *lines) { return count_lines(lines); }

sp_status spline_project_fwd(const sp_grid *grid, const float *coef, const sp_lines *lines,
                             float *sino, void *stream)
{
    g_err.clear();
    spx::GridDev g;
    spx::LinesDev L;
    sp_status st = check_grid(grid, &g);
    if (st != SP_OK) return st;
    if ((st = check_lines(lines, &L)) != SP_OK) return st;
    if (L.m == 0) return SP_OK;
    if (!coef || !sino) return fail(SP_EINVAL, "coef/sino pointers are NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    spx::LineHdr *hdr;
    float *tabs;
    void *extra = nullptr;
    if ((st = prepare(g, L, s, &hdr, &tabs, &extra)) != SP_OK) return st;
    cudaError_t e = run_fwd(g, L, hdr, tabs, extra, coef, sino, s);
    if (e != cudaSuccess) return cuda_fail(e, "forward projection");
    return SP_OK;
}

sp_status spline_project_adj(const sp_grid *grid, const float *sino, const sp_lines *lines,
                             float *coef_out, void *stream)
{
    g_err.clear();
    spx::GridDev g;
    spx::LinesDev L;
    sp_status st = check_grid(grid, &g);
    if (st != SP_OK) return st;
    if ((st = check_lines(lines, &L)) != SP_OK) return st;
    if (!coef_out) return fail(SP_EINVAL, "coef_out pointer is NULL");
    if (L.m > 0 && !sino) return fail(SP_EINVAL, "sino pointer is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (L.m == 0) {
        cudaError_t e = cudaMemsetAsync(coef_out, 0, sizeof(float) * (size_t)g.nx * g.ny, s);
        return e == cudaSuccess ? SP_OK : cuda_fail(e, "cudaMemsetAsync");
    }
    spx::LineHdr *hdr;
    float *tabs;
    void *extra = nullptr;
    if ((st = prepare(g, L, s, &hdr, &tabs, &extra)) != SP_OK) return st;
    cudaError_t e = run_adj(g, L, hdr, tabs, extra, sino, coef_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint projection");
    return SP_OK;
}

sp_status spline_lines_expand(const sp_lines *lines, float *theta_out, float *y_out, void *stream)
{
    g_err.clear();
    spx::LinesDev L;
    sp_status st = check_lines(lines, &L);
    if (st != SP_OK) return st;
    cudaError_t e = spx::launch_expand(L, theta_out, y_out, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SP_OK : cuda_fail(e, "line expansion");
}

sp_status spline_footprint_eval(const sp_grid *grid, int64_t count, const float *theta, const float *yt,
                                float *out, void *stream)
{
    g_err.clear();
    if (!grid) return fail(SP_EINVAL, "grid is NULL");
    sp_grid gg = *grid;
    gg.nx = gg.ny = 1;
    gg.h = 1.f;
    gg.cx = gg.cy = 0.f;
    spx::GridDev g;
    sp_status st0 = check_grid(&gg, &g);
    if (st0 != SP_OK) return st0;
    if (count < 0) return fail(SP_EINVAL, "count must be >= 0");
    if (count == 0) return SP_OK;
    if (!theta || !yt || !out) return fail(SP_EINVAL, "NULL pointer");
    void *ws = nullptr;
    sp_status st = workspace(sizeof(float) * (size_t)spx::kTabFloats * (size_t)count, &ws);
    if (st != SP_OK) return st;
    cudaError_t e = spx::launch_footprint_eval(g, count, theta, yt, out, static_cast<float *>(ws),
                                               static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SP_OK : cuda_fail(e, "footprint evaluation");
}

sp_status spline_visited(const sp_grid *grid, const sp_lines *lines, int32_t *counts,
                         const int64_t *offsets, int32_t *nodes, void *stream)
{
    g_err.clear();
    spx::GridDev g;
    spx::LinesDev L;
    sp_status st = check_grid(grid, &g);
    if (st != SP_OK) return st;
    if ((st = check_lines(lines, &L)) != SP_OK) return st;
    if (L.m == 0) return SP_OK;
    if (!counts) return fail(SP_EINVAL, "counts pointer is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    spx::LineHdr *hdr;
    float *tabs;
    if ((st = prepare(g, L, s, &hdr, &tabs)) != SP_OK) return st;
    cudaError_t e = spx::launch_visited(g, hdr, tabs, L.m, counts, offsets, nodes, s);
    return e == cudaSuccess ? SP_OK : cuda_fail(e, "visited set");
}

struct sp_plan {
    spx::GridDev g;
    spx::LinesDev L;
    int device;
    void *mem;
    spx::LineHdr *hdr;
    float *tabs;
    void *extra;       // strip scratch (transposed coefficients, slow-row counter) or NULL
    spx::StripRec rec; // row records written by prepare (base NULL: none)
    bool prepared;
    void *cg_ws;       // CGLS vectors and scalars, allocated on first use
    size_t cg_bytes;
    int path_fwd, path_adj;   // KernelPath of each direction
};

}  // extern "C"

namespace {
// Row records for the plan if it can keep them (see rec_bytes_wanted); false
// if it keeps none (the projections then traverse the rows themselves).
bool plan_alloc_records(sp_plan *p)
{
    if (p->rec.base) return true;
    const size_t rb = rec_bytes_wanted(p->g, p->L);
    if (rb == 0) return false;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess || rb > fr / 4 || rb > kRecMaxBytes) {
        cudaGetLastError();
        return false;
    }
    void *r = nullptr;
    if (cudaMalloc(&r, rb) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    p->rec = spx::StripRec{static_cast<unsigned char *>(r), spx::strip_rec_line_bytes(p->g)};
    return true;
}

sp_status plan_create(const sp_grid *grid, const sp_lines *lines, sp_plan **plan, bool keep_records)
{
    g_err.clear();
    if (!plan) return fail(SP_EINVAL, "plan is NULL");
    *plan = nullptr;
    spx::GridDev g;
    spx::LinesDev L;
    sp_status st = check_grid(grid, &g);
    if (st != SP_OK) return st;
    if ((st = check_lines(lines, &L)) != SP_OK) return st;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    size_t hb = align_up(sizeof(spx::LineHdr) * (size_t)L.m);
    size_t tb = align_up(sizeof(float) * (size_t)spx::kTabFloats * (size_t)table_count(L));
    size_t xb = align_up(extra_bytes(g, L));
    void *mem = nullptr;
    if (hb + tb + xb > 0) {
        e = cudaMalloc(&mem, hb + tb + xb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SP_ENOMEM, std::string("plan allocation failed: ") + cudaGetErrorString(e));
        }
    }
    sp_plan *p = new sp_plan;
    p->g = g;
    p->L = L;
    p->device = dev;
    p->mem = mem;
    p->hdr = reinterpret_cast<spx::LineHdr *>(mem);
    p->tabs = mem ? reinterpret_cast<float *>(static_cast<char *>(mem) + hb) : nullptr;
    p->extra = (mem && xb) ? static_cast<char *>(mem) + hb + tb : nullptr;
    p->L.order = static_cast<const int *>(order_area(g, L, p->extra));   // written by prepare
    p->prepared = false;
    p->cg_ws = nullptr;
    p->cg_bytes = 0;
    p->path_fwd = p->path_adj = kPathAuto;
    p->rec = spx::StripRec{nullptr, 0};
    if (p->extra) {
        e = cudaMemset(slow_counter(g, p->extra), 0, sizeof(int));
        if (e != cudaSuccess) {
            cudaFree(mem);
            delete p;
            return cuda_fail(e, "cudaMemset");
        }
    }
    if (keep_records) plan_alloc_records(p);
    *plan = p;
    return SP_OK;
}

// The plan's row records, if it keeps them (written by every prepare).
const spx::StripRec *plan_rec(const sp_plan *p) { return p->rec.base ? &p->rec : nullptr; }
}  // namespace

extern "C" {

sp_status spline_plan_create(const sp_grid *grid, const sp_lines *lines, sp_plan **plan)
{
    return plan_create(grid, lines, plan, false);
}

sp_status spline_plan_set_records(sp_plan *plan, int32_t keep)
{
    g_err.clear();
    if (!plan) return fail(SP_EINVAL, "plan is NULL");
    if (keep != 0 && keep != 1) return fail(SP_EINVAL, "keep must be 0 or 1");
    if (keep == 0) {
        if (plan->rec.base) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            cudaFree(plan->rec.base);
            plan->rec = spx::StripRec{nullptr, 0};
        }
        return SP_OK;
    }
    if (plan->rec.base) return SP_OK;
    if (rec_bytes_wanted(plan->g, plan->L) == 0)
        return fail(SP_EUNSUPPORTED, "row records exist only for B-spline or box-spline grids of degree >= 1");
    if (!plan_alloc_records(plan)) return fail(SP_ENOMEM, "row records do not fit in device memory");
    plan->prepared = false;   // records are written by the next prepare
    return SP_OK;
}

sp_status spline_plan_prepare(sp_plan *plan, void *stream)
{
    g_err.clear();
    if (!plan) return fail(SP_EINVAL, "plan is NULL");
    if (plan->L.m == 0) { plan->prepared = true; return SP_OK; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = spx::launch_prepare(plan->g, plan->L, plan->hdr, plan->tabs, table_count(plan->L), s);
    if (e != cudaSuccess) return cuda_fail(e, "line setup and footprint tables");
    if (plan->L.order) {
        e = spx::launch_line_order(plan->g, plan->L, plan->hdr, const_cast<int *>(plan->L.order), s);
        if (e != cudaSuccess) return cuda_fail(e, "line order");
    }
    if (plan->rec.base) {
        e = spx::launch_strip_record(plan->g, plan->L, plan->hdr, plan->tabs, plan->rec, s);
        if (e != cudaSuccess) return cuda_fail(e, "row records");
    }
    plan->prepared = true;
    return SP_OK;
}

sp_status spline_plan_fwd(const sp_plan *plan, const float *coef, float *sino, void *stream)
{
    g_err.clear();
    if (!plan) return fail(SP_EINVAL, "plan is NULL");
    if (!plan->prepared) return fail(SP_EINVAL, "plan not prepared");
    if (plan->L.m == 0) return SP_OK;
    if (!coef || !sino) return fail(SP_EINVAL, "coef/sino pointers are NULL");
    cudaError_t e = run_fwd(plan->g, plan->L, plan->hdr, plan->tabs, plan->extra, coef, sino,
                            static_cast<cudaStream_t>(stream), plan->path_fwd, plan_rec(plan));
    return e == cudaSuccess ? SP_OK : cuda_fail(e, "forward projection");
}

sp_status spline_plan_adj(const sp_plan *plan, const float *sino, float *coef_out, void *stream)
{
    g_err.clear();
    if (!plan) return fail(SP_EINVAL, "plan is NULL");
    if (!plan->prepared) return fail(SP_EINVAL, "plan not prepared");
    if (!coef_out) return fail(SP_EINVAL, "coef_out pointer is NULL");
    if (plan->L.m > 0 && !sino) return fail(SP_EINVAL, "sino pointer is NULL");
    cudaError_t e = run_adj(plan->g, plan->L, plan->hdr, plan->tabs, plan->extra, sino, coef_out,
                            static_cast<cudaStream_t>(stream), plan->path_adj, plan_rec(plan));
    return e == cudaSuccess ? SP_OK : cuda_fail(e, "adjoint projection");
}

namespace {
cudaError_t plan_fwd_cb(void *ctx, const float *coef, float *sino, cudaStream_t s)
{
    const sp_plan *p = static_cast<const sp_plan *>(ctx);
    return run_fwd(p->g, p->L, p->hdr, p->tabs, p->extra, coef, sino, s, p->path_fwd, plan_rec(p));
}
cudaError_t plan_adj_cb(void *ctx, const float *sino, float *coef_out, cudaStream_t s)
{
    const sp_plan *p = static_cast<const sp_plan *>(ctx);
    return run_adj(p->g, p->L, p->hdr, p->tabs, p->extra, sino, coef_out, s, p->path_adj, plan_rec(p));
}
}  // namespace

sp_status spline_plan_cgls(sp_plan *plan, const float *b, float *x, int32_t iters, double *gamma_hist,
                           void *stream)
{
    g_err.clear();
    if (!plan) return fail(SP_EINVAL, "plan is NULL");
    if (!plan->prepared) return fail(SP_EINVAL, "plan not prepared");
    if (!x) return fail(SP_EINVAL, "x pointer is NULL");
    if (plan->L.m > 0 && !b) return fail(SP_EINVAL, "b pointer is NULL");
    if (iters < 0) return fail(SP_EINVAL, "iters must be >= 0");
    const int64_t n = (int64_t)plan->g.nx * plan->g.ny, m = plan->L.m;
    const size_t need = spx::cg_workspace_bytes(n, m);
    if (plan->cg_bytes < need) {
        if (plan->cg_ws) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            cudaFree(plan->cg_ws);
            plan->cg_ws = nullptr;
            plan->cg_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&plan->cg_ws, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            plan->cg_ws = nullptr;
            return fail(SP_ENOMEM, std::string("CGLS workspace allocation failed: ") + cudaGetErrorString(e));
        }
        plan->cg_bytes = need;
    }
    spx::CgOps ops{plan, plan_fwd_cb, plan_adj_cb};
    cudaError_t e = spx::run_cgls(ops, n, m, b, x, iters, gamma_hist, plan->cg_ws, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SP_OK : cuda_fail(e, "CGLS");
}

int64_t spline_plan_lines(const sp_plan *plan) { return plan ? plan->L.m : -1; }

int64_t spline_plan_record_bytes(const sp_plan *plan)
{
    if (!plan) return -1;
    return plan->rec.base ? plan->L.m * (int64_t)plan->rec.line_bytes : 0;
}

}  // extern "C"

namespace {
// Mean device time of `reps` runs of f on stream s (after one untimed run).
template <typename F>
cudaError_t time_runs(F f, int reps, cudaStream_t s, float *ms)
{
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
    if ((e = f()) == cudaSuccess && (e = cudaEventRecord(a, s)) == cudaSuccess) {
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = f();
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
        if (e == cudaSuccess) *ms /= (float)reps;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}
}  // namespace

extern "C" {

sp_status spline_plan_set_paths(sp_plan *plan, int32_t fwd_path, int32_t adj_path)
{
    g_err.clear();
    if (!plan) return fail(SP_EINVAL, "plan is NULL");
    if (fwd_path < 0 || fwd_path > 2 || adj_path < 0 || adj_path > 3)
        return fail(SP_EINVAL, "path must be 0, 1 or 2 (the adjoint also 3)");
    plan->path_fwd = fwd_path;
    plan->path_adj = adj_path;
    return SP_OK;
}

sp_status spline_plan_autotune(sp_plan *plan, const float *coef, const float *sino, void *stream,
                               int32_t *fwd_path, int32_t *adj_path, float *ms_out)
{
    g_err.clear();
    if (!plan) return fail(SP_EINVAL, "plan is NULL");
    if (!plan->prepared) return fail(SP_EINVAL, "plan not prepared");
    const int64_t n = (int64_t)plan->g.nx * plan->g.ny, m = plan->L.m;
    if (m > 0 && (!coef || !sino)) return fail(SP_EINVAL, "coef/sino pointers are NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool both = plan->extra && spx::strip_supported(plan->g, plan->L) && m > 0;
    // fwd strip, fwd general, adj strip, adj general, adj gather
    float t[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int bf = both ? kPathStrip : kPathGeneral, ba = bf;
    const bool gather = both && spx::gather_supported(plan->g, plan->L);
    if (both) {
        float *tmp_s = nullptr, *tmp_c = nullptr;
        cudaError_t e = cudaMalloc(&tmp_s, sizeof(float) * (size_t)m);
        if (e == cudaSuccess) e = cudaMalloc(&tmp_c, sizeof(float) * (size_t)n);
        const spx::StripRec *rec = plan_rec(plan);
        for (int k = 0; k < (gather ? 5 : 4) && e == cudaSuccess; ++k) {
            const int path = k == 4 ? kPathGather : ((k & 1) ? kPathGeneral : kPathStrip);
            if (k < 2)
                e = time_runs([&] { return run_fwd(plan->g, plan->L, plan->hdr, plan->tabs, plan->extra, coef, tmp_s, s,
                                                   path, rec); },
                              3, s, &t[k]);
            else
                e = time_runs([&] { return run_adj(plan->g, plan->L, plan->hdr, plan->tabs, plan->extra, sino, tmp_c, s,
                                                   path, rec); },
                              3, s, &t[k]);
        }
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (tmp_s) cudaFree(tmp_s);
        if (tmp_c) cudaFree(tmp_c);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) return cuda_fail(e, "autotune");
        bf = t[0] <= t[1] ? kPathStrip : kPathGeneral;
        ba = t[2] <= t[3] ? kPathStrip : kPathGeneral;
        if (gather && t[4] < (ba == kPathStrip ? t[2] : t[3])) ba = kPathGather;
    }
    plan->path_fwd = bf;
    plan->path_adj = ba;
    if (fwd_path) *fwd_path = bf;
    if (adj_path) *adj_path = ba;
    if (ms_out) for (int k = 0; k < 5; ++k) ms_out[k] = t[k];
    return SP_OK;
}

// ------------------------------------------------------------------ batches
// A batch is a set of plans run together: each call forks the instances over
// internal streams and joins them back on the caller's stream, recorded once
// as a CUDA graph per set of data pointers and replayed afterwards.
}  // extern "C"

namespace {
constexpr int kBatchStreams = 8;

struct GraphCache {
    std::vector<const void *> key;
    cudaGraphExec_t exec = nullptr;
    void clear()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
    }
};
}  // namespace

extern "C" {

struct sp_batch {
    std::vector<sp_plan *> plans;
    cudaStream_t cap = nullptr;                 // capture origin
    cudaStream_t streams[kBatchStreams] = {};
    cudaEvent_t fork = nullptr, join[kBatchStreams] = {};
    GraphCache gfwd, gadj;
    // strip-kernel instances run as one persistent launch over a work queue
    spx::StripJob *jobs_dev[2] = {nullptr, nullptr};   // forward, adjoint
    std::vector<spx::StripJob> jobs_host[2];
    int64_t chunks[2] = {0, 0};
    // jobs grouped by kernel degree (one queue launch per degree):
    // jobs [gjob0, gjob0 + gnjob) of group deg own gtotal chunks
    int gjob0[2][4] = {}, gnjob[2][4] = {};
    int64_t gtotal[2][4] = {};
    unsigned long long *counter = nullptr;              // [2][4 degrees][3]: queue counters
    long long *defer = nullptr;                          // adjoint chunks deferred to float strips
    int64_t defer_cap = 0;
};

}  // extern "C"

namespace {
void batch_free(sp_batch *b)
{
    if (!b) return;
    b->gfwd.clear();
    b->gadj.clear();
    for (int k = 0; k < kBatchStreams; ++k) {
        if (b->streams[k]) cudaStreamDestroy(b->streams[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int d = 0; d < 2; ++d)
        if (b->jobs_dev[d]) cudaFree(b->jobs_dev[d]);
    if (b->counter) cudaFree(b->counter);
    if (b->defer) cudaFree(b->defer);
    for (sp_plan *p : b->plans) spline_plan_destroy(p);
    delete b;
}

// Fork the instances over the internal streams from `origin`, run op(i, s)
// for instance i and orig(origin) on the origin itself, and join back on
// `origin`.
template <typename Op, typename Orig>
cudaError_t fork_join(sp_batch *b, cudaStream_t origin, Op op, Orig orig)
{
    cudaError_t e = cudaEventRecord(b->fork, origin);
    for (int k = 0; k < kBatchStreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->streams[k], b->fork, 0);
    for (size_t i = 0; i < b->plans.size() && e == cudaSuccess; ++i) e = op(i, b->streams[i % kBatchStreams]);
    if (e == cudaSuccess) e = orig(origin);
    for (int k = 0; k < kBatchStreams && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->join[k], b->streams[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, b->join[k], 0);
    }
    return e;
}

// Replay the cached graph for these pointers, or capture a new one: set_up()
// runs first (host side, outside the capture), then fork_join(op, orig) is
// captured.
template <typename Op, typename SetUp, typename Orig>
cudaError_t run_graph(sp_batch *b, GraphCache &gc, const std::vector<const void *> &key, cudaStream_t s, Op op,
                      SetUp set_up, Orig orig)
{
    if (!gc.exec || gc.key != key) {
        gc.clear();
        cudaError_t e = set_up();
        if (e != cudaSuccess) return e;
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t eop = fork_join(b, b->cap, op, orig);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->cap, &graph);
        if (eop != cudaSuccess) e = eop;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gc.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            gc.exec = nullptr;
            return e;
        }
        gc.key = key;
    }
    return cudaGraphLaunch(gc.exec, s);
}

// Queue entries of the instances of direction d (0 forward, 1 adjoint) that
// run on the strip kernels, uploaded to the batch's job array.  Runs outside
// any capture; the device is synchronised first because a graph recorded
// earlier may still read the previous array.
template <typename In, typename Out>
cudaError_t upload_jobs(sp_batch *b, int d, In in, Out outp, std::vector<char> &queued)
{
    std::vector<spx::StripJob> &hj = b->jobs_host[d];
    hj.clear();
    queued.assign(b->plans.size(), 0);
    int64_t all = 0;
    for (int deg = 0; deg <= 3; ++deg) {
        b->gjob0[d][deg] = (int)hj.size();
        int64_t c0 = 0;   // chunk indices count within the degree's group
        for (size_t i = 0; i < b->plans.size(); ++i) {
            const sp_plan *p = b->plans[i];
            const int path = d ? p->path_adj : p->path_fwd;
            // (degree 0 takes the strip kernels when set or tuned to them)
            if (p->g.kdeg != deg || p->L.m == 0 || !use_strip(p->g, p->L, p->extra, path)) continue;
            spx::StripJob J = d ? spx::make_strip_job(p->g, p->L, p->hdr, p->tabs, true, nullptr,
                                                      const_cast<float *>(in[i]), outp[i], p->extra,
                                                      slow_counter(p->g, p->extra))
                                : spx::make_strip_job(p->g, p->L, p->hdr, p->tabs, false, in[i], outp[i], nullptr,
                                                      p->extra, slow_counter(p->g, p->extra));
            J.chunk0 = c0;
            c0 += spx::strip_job_chunks(J);
            hj.push_back(J);
            queued[i] = 1;
        }
        b->gnjob[d][deg] = (int)hj.size() - b->gjob0[d][deg];
        b->gtotal[d][deg] = c0;
        all += c0;
    }
    const int64_t c0 = all;
    b->chunks[d] = c0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && d == 1 && c0 > b->defer_cap) {
        if (b->defer) cudaFree(b->defer);
        b->defer = nullptr;
        b->defer_cap = 0;
        e = cudaMalloc(&b->defer, sizeof(long long) * (size_t)c0);
        if (e == cudaSuccess) b->defer_cap = c0;
    }
    if (e == cudaSuccess && !hj.empty())
        e = cudaMemcpy(b->jobs_dev[d], hj.data(), sizeof(spx::StripJob) * hj.size(), cudaMemcpyHostToDevice);
    return e;
}

// The queued instances on the capture origin: per-instance set-up, the
// persistent kernel, per-instance completion.
cudaError_t run_queue(sp_batch *b, int d, cudaStream_t s)
{
    const std::vector<spx::StripJob> &hj = b->jobs_host[d];
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < hj.size() && e == cudaSuccess; ++k) e = spx::launch_strip_pre(hj[k], d == 1, s);
    int64_t defer0 = 0;   // each degree's deferred chunks in its own part of the list
    for (int deg = 0; deg <= 3 && e == cudaSuccess; ++deg) {
        if (b->gnjob[d][deg] == 0) continue;
        e = spx::launch_strip_queue(deg, d == 1, b->jobs_dev[d] + b->gjob0[d][deg], b->gnjob[d][deg],
                                    b->gtotal[d][deg], b->counter + 12 * d + 3 * deg,
                                    d == 1 ? b->defer + defer0 : nullptr, s);
        defer0 += b->gtotal[d][deg];
    }
    for (size_t k = 0; k < hj.size() && e == cudaSuccess; ++k) e = spx::launch_strip_post(hj[k], d == 1, s);
    return e;
}
}  // namespace

extern "C" {

sp_status spline_batch_create(int32_t count, const sp_grid *grids, const sp_lines *lines, sp_batch **batch)
{
    g_err.clear();
    if (!batch) return fail(SP_EINVAL, "batch is NULL");
    *batch = nullptr;
    if (count < 1) return fail(SP_EINVAL, "count must be >= 1");
    if (!grids || !lines) return fail(SP_EINVAL, "grids/lines are NULL");
    sp_batch *b = new sp_batch;
    for (int32_t i = 0; i < count; ++i) {
        sp_plan *p = nullptr;
        sp_status st = plan_create(grids + i, lines + i, &p, false);
        if (st != SP_OK) {
            std::string msg = "instance " + std::to_string(i) + ": " + g_err;
            batch_free(b);
            return fail(st, msg);
        }
        b->plans.push_back(p);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int d = 0; d < 2 && e == cudaSuccess; ++d) e = cudaMalloc(&b->jobs_dev[d], sizeof(spx::StripJob) * (size_t)count);
    if (e == cudaSuccess) e = cudaMalloc(&b->counter, 24 * sizeof(unsigned long long));
    for (int k = 0; k < kBatchStreams && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch streams");
    }
    *batch = b;
    return SP_OK;
}

sp_status spline_batch_prepare(sp_batch *batch, void *stream)
{
    g_err.clear();
    if (!batch) return fail(SP_EINVAL, "batch is NULL");
    sp_status st = SP_OK;
    cudaError_t e = fork_join(batch, static_cast<cudaStream_t>(stream), [&](size_t i, cudaStream_t s) {
        st = spline_plan_prepare(batch->plans[i], s);
        return st == SP_OK ? cudaSuccess : cudaErrorUnknown;
    }, [](cudaStream_t) { return cudaSuccess; });
    if (st != SP_OK) return st;
    return e == cudaSuccess ? SP_OK : cuda_fail(e, "batch prepare");
}

sp_status spline_batch_fwd(sp_batch *batch, const float *const *coef, float *const *sino, void *stream)
{
    g_err.clear();
    if (!batch || !coef || !sino) return fail(SP_EINVAL, "NULL argument");
    std::vector<const void *> key;
    for (size_t i = 0; i < batch->plans.size(); ++i) {
        const sp_plan *p = batch->plans[i];
        if (!p->prepared) return fail(SP_EINVAL, "instance " + std::to_string(i) + " not prepared");
        if (p->L.m > 0 && (!coef[i] || !sino[i])) return fail(SP_EINVAL, "NULL pointer of instance " + std::to_string(i));
        key.push_back(coef[i]);
        key.push_back(sino[i]);
    }
    std::vector<char> queued;
    cudaError_t e = run_graph(
        batch, batch->gfwd, key, static_cast<cudaStream_t>(stream),
        [&](size_t i, cudaStream_t s) {
            const sp_plan *p = batch->plans[i];
            if (p->L.m == 0 || queued[i]) return cudaSuccess;
            return run_fwd(p->g, p->L, p->hdr, p->tabs, p->extra, coef[i], sino[i], s, p->path_fwd);
        },
        [&] { return upload_jobs(batch, 0, coef, sino, queued); },
        [&](cudaStream_t s) { return run_queue(batch, 0, s); });
    return e == cudaSuccess ? SP_OK : cuda_fail(e, "batch forward");
}

sp_status spline_batch_adj(sp_batch *batch, const float *const *sino, float *const *coef_out, void *stream)
{
    g_err.clear();
    if (!batch || !sino || !coef_out) return fail(SP_EINVAL, "NULL argument");
    std::vector<const void *> key;
    for (size_t i = 0; i < batch->plans.size(); ++i) {
        const sp_plan *p = batch->plans[i];
        if (!p->prepared) return fail(SP_EINVAL, "instance " + std::to_string(i) + " not prepared");
        if (!coef_out[i] || (p->L.m > 0 && !sino[i])) return fail(SP_EINVAL, "NULL pointer of instance " + std::to_string(i));
        key.push_back(sino[i]);
        key.push_back(coef_out[i]);
    }
    std::vector<char> queued;
    cudaError_t e = run_graph(
        batch, batch->gadj, key, static_cast<cudaStream_t>(stream),
        [&](size_t i, cudaStream_t s) {
            const sp_plan *p = batch->plans[i];
            if (queued[i]) return cudaSuccess;
            return run_adj(p->g, p->L, p->hdr, p->tabs, p->extra, sino[i], coef_out[i], s, p->path_adj);
        },
        [&] { return upload_jobs(batch, 1, sino, coef_out, queued); },
        [&](cudaStream_t s) { return run_queue(batch, 1, s); });
    return e == cudaSuccess ? SP_OK : cuda_fail(e, "batch adjoint");
}

sp_status spline_batch_autotune(sp_batch *batch, const float *const *coef, const float *const *sino, void *stream,
                                int32_t *paths)
{
    g_err.clear();
    if (!batch || !coef || !sino) return fail(SP_EINVAL, "NULL argument");
    const size_t cnt = batch->plans.size();
    for (size_t i = 0; i < cnt; ++i) {
        sp_status st = spline_plan_autotune(batch->plans[i], coef[i], sino[i], stream, nullptr, nullptr, nullptr);
        if (st != SP_OK) return fail(st, "instance " + std::to_string(i) + ": " + g_err);
    }
    // Whole batch: the instances' own choices against the strip kernels
    // wherever they apply.  Inside the shared queue launch a small instance
    // fills no GPU on its own, so timing it alone can understate the strip
    // kernels.  Outputs go to temporary buffers.
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t ms_tot = 0, ns_tot = 0;
    std::vector<char> eligible(cnt, 0);
    for (size_t i = 0; i < cnt; ++i) {
        const sp_plan *p = batch->plans[i];
        ms_tot += align_up(sizeof(float) * (size_t)p->L.m);
        ns_tot += align_up(sizeof(float) * (size_t)p->g.nx * p->g.ny);
        eligible[i] = p->extra && spx::strip_supported(p->g, p->L) && p->L.m > 0;
    }
    char *tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, ms_tot + ns_tot);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    std::vector<float *> ts(cnt), tc(cnt);
    {
        size_t o = 0;
        for (size_t i = 0; i < cnt; ++i) {
            ts[i] = reinterpret_cast<float *>(tmp + o);
            o += align_up(sizeof(float) * (size_t)batch->plans[i]->L.m);
        }
        for (size_t i = 0; i < cnt; ++i) {
            tc[i] = reinterpret_cast<float *>(tmp + o);
            o += align_up(sizeof(float) * (size_t)batch->plans[i]->g.nx * batch->plans[i]->g.ny);
        }
    }
    sp_status st = SP_OK;
    for (int d = 0; d < 2 && st == SP_OK && e == cudaSuccess; ++d) {
        std::vector<int> own(cnt);
        bool differs = false;
        for (size_t i = 0; i < cnt; ++i) {
            own[i] = d ? batch->plans[i]->path_adj : batch->plans[i]->path_fwd;
            differs = differs || (eligible[i] && own[i] != kPathStrip);
        }
        if (!differs) continue;
        float t[2] = {0.f, 0.f};   // own choices, strip wherever it applies
        for (int v = 0; v < 2 && st == SP_OK && e == cudaSuccess; ++v) {
            for (size_t i = 0; i < cnt; ++i) {
                int &path = d ? batch->plans[i]->path_adj : batch->plans[i]->path_fwd;
                path = (v == 1 && eligible[i]) ? kPathStrip : own[i];
            }
            batch->gfwd.clear();
            batch->gadj.clear();
            e = time_runs([&] {
                st = d ? spline_batch_adj(batch, sino, tc.data(), stream)
                       : spline_batch_fwd(batch, coef, ts.data(), stream);
                return st == SP_OK ? cudaSuccess : cudaErrorUnknown;
            }, 3, s, &t[v]);
        }
        if (st == SP_OK && e == cudaSuccess && t[0] <= t[1])
            for (size_t i = 0; i < cnt; ++i) (d ? batch->plans[i]->path_adj : batch->plans[i]->path_fwd) = own[i];
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    batch->gfwd.clear();
    batch->gadj.clear();
    for (int d = 0; d < 2; ++d) {   // the timing runs' queues; the next call records anew
        batch->jobs_host[d].clear();
        batch->chunks[d] = 0;
    }
    cudaFree(tmp);
    if (st != SP_OK) return fail(st, "batch autotune: " + g_err);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
    if (paths)
        for (size_t i = 0; i < cnt; ++i) {
            paths[2 * i] = batch->plans[i]->path_fwd;
            paths[2 * i + 1] = batch->plans[i]->path_adj;
        }
    return SP_OK;
}

int32_t spline_batch_count(const sp_batch *batch) { return batch ? (int32_t)batch->plans.size() : -1; }

int32_t spline_batch_queued(const sp_batch *batch, int32_t adjoint)
{
    if (!batch) return -1;
    return (int32_t)batch->jobs_host[adjoint ? 1 : 0].size();
}

sp_status spline_batch_destroy(sp_batch *batch)
{
    g_err.clear();
    if (!batch) return SP_OK;
    cudaError_t e = cudaDeviceSynchronize();
    batch_free(batch);
    return e == cudaSuccess ? SP_OK : cuda_fail(e, "cudaDeviceSynchronize");
}

sp_status spline_plan_stats(const sp_plan *plan, int64_t *slow_rows)
{
    g_err.clear();
    if (!plan || !slow_rows) return fail(SP_EINVAL, "NULL argument");
    *slow_rows = 0;
    if (!plan->extra) return SP_OK;
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, slow_counter(plan->g, plan->extra), sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    *slow_rows = v;
    return SP_OK;
}

sp_status spline_plan_destroy(sp_plan *plan)
{
    g_err.clear();
    if (!plan) return SP_OK;
    sp_status st = SP_OK;
    if (plan->mem || plan->cg_ws || plan->rec.base) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(e, "cudaDeviceSynchronize");
        if (plan->mem) cudaFree(plan->mem);
        if (plan->cg_ws) cudaFree(plan->cg_ws);
        if (plan->rec.base) cudaFree(plan->rec.base);
    }
    delete plan;
    return st;
}

sp_status sp_release_workspace(void)
{
    g_err.clear();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return SP_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace &ws = g_ws[dev];
    if (ws.ptr) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
        cudaFree(ws.ptr);
    }
    ws.ptr = nullptr;
    ws.bytes = 0;
    return SP_OK;
}

const char *sp_last_error(void) { return g_err.c_str(); }

int32_t sp_version(void) { return 100; }

sp_status sp_fp32_peak(int32_t packed, double *tflops, float *ms, void *stream)
{
    g_err.clear();
    if (packed != 0 && packed != 1) return fail(SP_EINVAL, "packed must be 0 or 1");
    if (!tflops) return fail(SP_EINVAL, "tflops is NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    const int blocks = 8 * sms, iters = 8192;   // 2048 threads per SM, ~10 ms
    void *ws = nullptr;
    sp_status st = workspace(sizeof(float) * 256 * (size_t)blocks, &ws);
    if (st != SP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    if (e == cudaSuccess) e = spx::launch_fp32_peak(packed, blocks, iters, static_cast<float *>(ws), s);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = spx::launch_fp32_peak(packed, blocks, iters, static_cast<float *>(ws), s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && (k == 0 || t < best)) best = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "FP32 peak probe");
    *tflops = (double)spx::fp32_peak_flops(packed, blocks, iters) / (1e-3 * (double)best) * 1e-12;
    if (ms) *ms = best;
    return SP_OK;
}

}  // extern "C"
