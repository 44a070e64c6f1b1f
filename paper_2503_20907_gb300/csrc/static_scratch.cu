// Forward projection without any device allocation.
//
// Some callers cannot let a library allocate device memory: programs that
// reserve the whole device up front for their own memory pool (a framework's
// caching allocator, a fixed-budget reconstruction service), where a foreign
// cudaMalloc fails or fragments the pool, and latency-bound pipelines that
// cannot afford the device-wide synchronisation that cudaFree (and growing a
// cached workspace) implies.  spline_project_fwd_noalloc serves them.  It
// gives the same result as spline_project_fwd, but always through the line
// setup, table and warp-per-line forward kernels: the strip kernels that
// spline_project_fwd takes for parallel and fan beams of degree >= 1 need a
// transposed copy of the image, which the fixed array does not hold, so this
// entry point runs at the speed of the warp-per-line path.  Its scratch
// (per-line records and footprint tables) lives in the fixed array below.
//
// When that array takes device memory: the library is built without
// relocatable device code, so the array sits in a module of its own, and
// under lazy module loading (CUDA_MODULE_LOADING=LAZY, which PyTorch turns
// on) the CUDA driver loads that module, and reserves the array's 48 MiB, only at
// the first cudaGetSymbolAddress on a device, i.e. during the first call of
// this entry point there.  That first call (a one-line list suffices) is
// therefore the one step that takes device memory; callers make it before
// they hand the rest of the device to their own pool and before any stream
// capture.  From then on the array stays until the process exits.
#include <mutex>
#include <string>

#include "common.cuh"

namespace spx {
sp_status check_grid_for(const sp_grid *g, GridDev *out);
sp_status check_lines_for(const sp_lines *L, LinesDev *out);
sp_status record_error(sp_status st, const std::string &msg);
void clear_error();
}  // namespace spx

namespace {

// 48 MiB of scratch per device for the per-line records (64 B per line) and
// the footprint tables (1312 B per line, or per view for parallel beams).
constexpr size_t kStaticScratchBytes = 48u << 20;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDev = 64;
std::mutex g_sym_mu;
void *g_sym_ptr[kMaxDev] = {};

// Device address of g_static_scratch on the current device.  In host code the
// name of a __device__ array is only a host-side stand-in, so the address has
// to be asked of the runtime, once per device, with that device current.
sp_status scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return spx::record_error(SP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDev) return spx::record_error(SP_EUNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_sym_mu);
    if (!g_sym_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return spx::record_error(SP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_sym_ptr[dev] = p;
    }
    *out = g_sym_ptr[dev];
    return SP_OK;
}

}  // namespace

extern "C" {

sp_status spline_project_fwd_noalloc(const sp_grid *grid, const float *coef, const sp_lines *lines,
                                     float *sino, void *stream)
{
    spx::clear_error();
    spx::GridDev g;
    spx::LinesDev L;
    sp_status st = spx::check_grid_for(grid, &g);
    if (st != SP_OK) return st;
    if ((st = spx::check_lines_for(lines, &L)) != SP_OK) return st;
    if (L.m == 0) return SP_OK;
    if (!coef || !sino) return spx::record_error(SP_EINVAL, "coef/sino pointers are NULL");
    const int64_t n_tab = L.kind == SP_LINES_PARALLEL ? (int64_t)L.n_view : L.m;
    const size_t hb = ((sizeof(spx::LineHdr) * (size_t)L.m) + 255) & ~(size_t)255;
    const size_t need = hb + sizeof(float) * (size_t)spx::kTabFloats * (size_t)n_tab;
    if (need > kStaticScratchBytes)
        return spx::record_error(SP_EINVAL, "line list needs " + std::to_string(need) +
                                           " bytes of scratch; the static scratch holds " +
                                           std::to_string(kStaticScratchBytes) +
                                           " (about 36,000 lines with their own footprint table)");
    void *base = nullptr;
    if ((st = scratch_address(&base)) != SP_OK) return st;
    spx::LineHdr *hdr = static_cast<spx::LineHdr *>(base);
    float *tabs = reinterpret_cast<float *>(static_cast<unsigned char *>(base) + hb);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Records and tables are written whole by the two set-up kernels before
    // the projection reads them, so nothing in the array needs clearing.
    cudaError_t e = spx::launch_setup(g, L, hdr, tabs, s);
    if (e == cudaSuccess) e = spx::launch_tables(g, L, tabs, n_tab, s);
    if (e == cudaSuccess) e = spx::launch_fwd(g, hdr, tabs, L.m, coef, sino, s);
    if (e != cudaSuccess) return spx::record_error(SP_ECUDA, std::string("forward projection: ") + cudaGetErrorString(e));
    return SP_OK;
}

}  // extern "C"
