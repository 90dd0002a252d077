// Preconditioner entry point that allocates nothing.
//
// epr_precondition needs a plan, and a plan allocates device memory (its
// workspace and twiddle tables) with cudaMalloc.  Some callers cannot let a
// library do that: applications whose device memory is all handed out by
// their own pool allocator, applications that fix their memory budget at
// start-up and must not grow it later, and latency-critical paths where a
// cudaMalloc, which may synchronise the device, is not acceptable.
// epr_precondition_noalloc serves them: it runs the same three kernels as
// epr_precondition (forward row FFT, column filter, inverse row FFT) but
// keeps its scratch -- the packed half spectrum and the two twiddle tables
// -- in one file-scope __device__ array of fixed size.  It calls no
// cudaMalloc, cudaFree or other allocating routine.
//
// That array exists on every GPU that loads this library, from module load
// until the process exits, whether or not the entry point is ever called.
// Every call uses the same array: two calls whose kernels overlap on a GPU
// (different streams, no ordering between them) race on it.  Nothing in it
// needs to start at zero -- each call writes the twiddles and the whole
// spectrum region it reads.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "epr_internal.cuh"

// Scratch: up to kNoallocPixels map pixels of half spectrum (4 bytes per
// pixel) plus the twiddle tables of the two axes.
namespace {
constexpr size_t kNoallocPixels = (size_t)4 << 20;                 // 4 Mi pixels
constexpr size_t kNoallocSpectrum = kNoallocPixels * 4;             // 16 MiB
constexpr size_t kNoallocTwiddles = (size_t)2 * 4096 * sizeof(float2);
constexpr size_t kNoallocBytes = kNoallocSpectrum + kNoallocTwiddles;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// launchers of the preconditioner passes (rowfft.cu, colfft.cu)
cudaError_t epr_launch_row_fwd(const EprConsts& C, const EprWork& W, int mode, const float* T,
                               const float* D, const float* G, int line0, int nl, int it,
                               float tol, int batch, int check_done, cudaStream_t stream);
cudaError_t epr_launch_row_inv(const EprConsts& C, const EprWork& W, int mode, float* Out,
                               int line0, int nl, int it, float omega, float eps, float tol,
                               int batch, int check_done, cudaStream_t stream);
cudaError_t epr_launch_col(const EprConsts& C, const EprWork& W, int line0, int nl, int batch,
                           int check_done, int cw_hint, int rho_it, cudaStream_t stream);
cudaError_t epr_row_init();
cudaError_t epr_col_init();

namespace {

// exp(-2 pi i t / n) for t < n, in double then rounded (the table a plan
// builds on the host), written into the scratch array
__global__ void k_noalloc_twiddles(float2* tw, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s, c;
    sincospi(-2.0 * (double)t / (double)n, &s, &c);
    tw[t] = make_float2((float)c, (float)s);
}

// Device address of the scratch array.  In host code the array's name is
// only a host-side stand-in, so the address is looked up with the device
// current, on every call (cudaGetSymbolAddress allocates nothing and is
// cheap).  The kernels' shared-memory attributes are set once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
bool g_attr_ready[kMaxDevices];

cudaError_t setup(int dev, unsigned char** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_attr_ready[dev]) {
        e = epr_row_init();
        if (e != cudaSuccess) return e;
        e = epr_col_init();
        if (e != cudaSuccess) return e;
        g_attr_ready[dev] = true;
    }
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

bool size_ok(int n)
{
    if (n < 16 || n > 4096) return false;
    int m = n, twos = 0;
    while (m % 2 == 0) {
        m /= 2;
        ++twos;
    }
    while (m % 3 == 0) m /= 3;
    return m == 1 && twos >= 3;
}

}  // namespace

extern "C" epr_status epr_precondition_noalloc(float* g, int nx, int ny, double pixel_m, double L_m,
                                               double energy_keV, double delta, double beta,
                                               int batch, void* stream)
{
    if (!g || batch <= 0 || !(pixel_m > 0.0) || !(L_m >= 0.0) || !(energy_keV > 0.0) ||
        !(beta > 0.0) || !isfinite(delta))
        return EPR_ERR_INVALID_ARG;
    if (((uintptr_t)g & 15u) != 0) return EPR_ERR_INVALID_ARG;
    if (!size_ok(nx) || !size_ok(ny)) return EPR_ERR_UNSUPPORTED_SIZE;
    if ((size_t)batch * nx * ny > kNoallocPixels) return EPR_ERR_UNSUPPORTED_SIZE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EPR_ERR_CUDA;
    unsigned char* base = nullptr;
    if (setup(dev, &base) != cudaSuccess) return EPR_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;

    // constants of one line, as a plan derives them
    const double kPi = 3.14159265358979323846;
    const double lam = 1.2398419843320026e-6 / (energy_keV * 1e3);
    const double k = 2.0 * kPi / lam, mu = 2.0 * k * beta, Ld = L_m * delta;
    EprConsts C = {};
    C.nx = nx;
    C.ny = ny;
    C.ns = 1;
    C.half = nx / 2;
    C.smax = 1;
    C.inv_n = (float)(1.0 / ((double)nx * ny));
    C.f[0] = 1.f;
    C.mu[0] = (float)mu;
    const double fx1 = 1.0 / (nx * pixel_m), fy1 = 1.0 / (ny * pixel_m);
    C.ha[0] = (float)(Ld * 4.0 * kPi * kPi * fx1 * fx1 / mu);
    C.hb[0] = (float)(Ld * 4.0 * kPi * kPi * fy1 * fy1 / mu);

    EprWork W = {};
    W.S = reinterpret_cast<float2*>(base);
    float2* tw_x = reinterpret_cast<float2*>(base + kNoallocSpectrum);
    float2* tw_y = tw_x + 4096;
    W.tw_x = tw_x;
    W.tw_y = tw_y;

    k_noalloc_twiddles<<<(nx + 255) / 256, 256, 0, s>>>(tw_x, nx);
    k_noalloc_twiddles<<<(ny + 255) / 256, 256, 0, s>>>(tw_y, ny);
    epr_count_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = epr_launch_row_fwd(C, W, 2, nullptr, nullptr, g, 0, 1, 0, 0.f, batch, 0, s);
    if (e == cudaSuccess) e = epr_launch_col(C, W, 0, 1, batch, 0, 0, -1, s);
    if (e == cudaSuccess) e = epr_launch_row_inv(C, W, 1, g, 0, 1, 0, 1.f, 0.f, 0.f, batch, 0, s);
    return e == cudaSuccess ? EPR_OK : EPR_ERR_CUDA;
}
