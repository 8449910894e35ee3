// A pressure solve that allocates no memory: the multigrid hierarchy, the
// coarsest-level factors and the reduction partials live in one file-scope
// device array of fixed size, and the host-side read-back goes to a static
// host array.  Callers pass only their inputs and outputs.
#include <string>
#include <vector>

#include "ib_internal.cuh"

namespace {

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[IB_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void *g_scratch_dev[kMaxDevices] = {};  // device address of the array, per device
double g_read_back[16];                 // host landing area of the norm read-back
ibk::MG g_mg;                           // views into the scratch array (no ownership)
std::string g_err;

}  // namespace

extern "C" const char *mg_solve_noalloc_error(void)
{
    return g_err.c_str();
}

extern "C" ib_status mg_solve_noalloc(int32_t nx, int32_t ny, double h, const double *bx,
                                      const double *by, const double *rhs, double *p,
                                      int precision, double tol, int max_cycles, int nu1,
                                      int nu2, int *cycles_out, double *relres_out,
                                      void *stream)
{
    if (nx < 2 || ny < 2 || (long)nx * ny > IB_NOALLOC_MAX_CELLS || !(h > 0) || !bx || !by ||
        !rhs || !p || precision < 0 || precision > 2 || !(tol >= 0) || max_cycles < 0 ||
        nu1 < 0 || nu2 < 0) {
        g_err = "bad argument (sizes, null pointer, precision outside 0..2, or more than "
                "IB_NOALLOC_MAX_CELLS cells)";
        return IB_EINVAL;
    }
    g_err.clear();
    std::vector<int> nxs, nys;
    if (!ibk::mg_levels(nx, ny, nxs, nys)) {
        g_err = "the grid does not coarsen to a small enough coarsest level";
        return IB_EINVAL;
    }
    const size_t need = ibk::mg_layout(g_mg, nx, ny, h, nullptr);
    if (need > (size_t)IB_NOALLOC_SCRATCH_BYTES) {
        g_err = "the multigrid hierarchy does not fit the scratch array";
        return IB_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        g_err = "no current CUDA device";
        return IB_ECUDA;
    }
    if (!g_scratch_dev[dev]) {
        // set-up on the first call on this device (with it current): the host
        // symbol is only a stand-in, kernels need the device address
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            g_err = "cudaGetSymbolAddress of the scratch array failed";
            return IB_ECUDA;
        }
        g_scratch_dev[dev] = ptr;
    }
    cudaStream_t s = (cudaStream_t)stream;
    ibk::mg_layout(g_mg, nx, ny, h, (char *)g_scratch_dev[dev]);
    g_mg.red_host = g_read_back;
    // the reduction's block counter and the control block (its fault word)
    // must start at zero; everything else in the scratch is written before it
    // is read
    if (cudaMemsetAsync(g_mg.red_count, 0, 64, s) != cudaSuccess ||
        cudaMemsetAsync(g_mg.ctl, 0, sizeof(ibk::SolveCtl), s) != cudaSuccess) {
        g_err = "clearing the scratch control block failed";
        return IB_ECUDA;
    }
    ibk::mg_build(g_mg, bx, by, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_err = cudaGetErrorString(e);
        return IB_ECUDA;
    }
    return ibk::mg_run_direct(g_mg, rhs, p, precision, tol, max_cycles, nu1, nu2, cycles_out,
                              relres_out, s, g_err);
}
