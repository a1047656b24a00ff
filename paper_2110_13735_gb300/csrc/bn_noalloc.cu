// bn_noalloc.cu -- evaluation of the 2-D collision operator without any device allocation.
//
// bn_eval_collision_device works in buffers that bn_create_solver allocated for the solver.
// This variant takes its working memory (transform buffer, modes, FP32 modes, per-CTA
// partial sums, combined modes, S(b) sums, the modes of the kernel-mode rounding correction, error
// flag) from one file-scope device array instead, so
// the call itself allocates nothing.  It is meant for callers that must not allocate at
// evaluation time -- code running where cudaMalloc/cudaFree are not allowed or not wanted
// (they synchronise the whole device, and fail when another allocator in the process has
// already reserved the memory) -- and that still want the operator of an existing solver,
// whose read-only kernel-mode tables, work lists and twiddles it uses.
//
// The array holds kNoAllocScratchBytes bytes on every device that loads the library, for
// the life of the process.  All calls in the process share it and it keeps the contents of
// the last call: every call clears what must start at zero (the error flag) and overwrites
// the rest, and calls whose GPU work overlaps in time race on it.
#include <cstdio>
#include <mutex>
#include <string>

#include "bn_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 12u << 20;   // 12 MiB: enough for every 2-D size (N <= 64)

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_na_mu;
void* g_na_ptr[64] = {};   // device address of the array, per device ordinal (set up once)

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the scratch array on device `dev`, which must be the current device; the
// first call on a device looks it up (host code may not take the address of a __device__
// variable directly: its host-side name is only a stand-in).
bn_status scratch_ptr(int dev, void** out) {
    if (dev < 0 || dev >= 64) {
        bn::set_last_error("device ordinal out of range for the no-allocation scratch");
        return BN_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            bn::set_last_error(std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e));
            return BN_ERR_CUDA;
        }
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return BN_OK;
}

}  // namespace

extern "C" {

bn_status bn_eval_collision_noalloc(const bn_solver* s, const double* f_dev, double* Q_dev, size_t count,
                                    void* cuda_stream) {
    if (!s || !f_dev || !Q_dev) {
        bn::set_last_error("null argument");
        return BN_ERR_ARG;
    }
    // the solver's tables and work lists live on s->device: the call must run there
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        bn::set_last_error("no usable CUDA device");
        return BN_ERR_CUDA;
    }
    if (cur != s->device) {
        bn::set_last_error("the current device is not the solver's device: make the solver's device current first");
        return BN_ERR_ARG;
    }
    if (s->g.d != 2 || s->nd) {
        bn::set_last_error("the no-allocation evaluation covers 2-D solvers with the LINEAR truncation only");
        return BN_ERR_UNSUPPORTED;
    }
    const size_t nm = (size_t)s->g.nModes;
    if (count != nm) {
        bn::set_last_error("count must be N^d");
        return BN_ERR_ARG;
    }
    // layout of the scratch array for this solver
    const int nPart = bn::fused2d_partials(s);
    const size_t o_err = 0;
    const size_t o_work = align256(o_err + sizeof(int) * 4);
    const size_t o_ghat = align256(o_work + nm * sizeof(double2));
    const size_t o_g32 = align256(o_ghat + nm * sizeof(double2));
    const size_t o_qhat = align256(o_g32 + nm * sizeof(float2));
    const size_t o_sb = align256(o_qhat + nm * sizeof(double2));
    const size_t o_qlo = align256(o_sb + (size_t)s->g.nExt * sizeof(float2));
    const size_t o_part = align256(o_qlo + nm * sizeof(double2));
    const size_t need = o_part + (size_t)nPart * nm * sizeof(double2);
    if (need > kNoAllocScratchBytes) {
        char buf[200];
        std::snprintf(buf, sizeof buf, "needs %zu bytes of scratch; the no-allocation scratch holds %zu", need,
                      kNoAllocScratchBytes);
        bn::set_last_error(std::string(buf));
        return BN_ERR_ARG;
    }
    void* base = nullptr;
    bn_status st = scratch_ptr(s->device, &base);
    if (st != BN_OK) return st;
    unsigned char* b = static_cast<unsigned char*>(base);
    int* err = reinterpret_cast<int*>(b + o_err);
    double2* work = reinterpret_cast<double2*>(b + o_work);
    double2* ghat = reinterpret_cast<double2*>(b + o_ghat);
    float2* g32 = reinterpret_cast<float2*>(b + o_g32);
    double2* qhat = reinterpret_cast<double2*>(b + o_qhat);
    double2* part = reinterpret_cast<double2*>(b + o_part);
    double2* qlo = reinterpret_cast<double2*>(b + o_qlo);
    void* sb = b + o_sb;
    const bool mixed = s->opt.precision == BN_MIXED;
    cudaStream_t strm = (cudaStream_t)cuda_stream;

    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), strm);   // the only state that must start at zero
    if (e == cudaSuccess) {
        bn::dft2_forward_into(s, strm, f_dev, work, ghat, mixed ? g32 : nullptr);
        const void* gin = mixed ? (const void*)g32 : (const void*)ghat;
        const bool lo = bn::beta_split_on(s);
        // the kernel-mode rounding correction: the residual-table pass first (into qlo), then the
        // main pass reuses the partials and S(b) scratch (stream order) and qlo is added to Q^
        if (lo) bn::fused2d_into(s, strm, gin, part, qlo, err, sb, true);
        bn::fused2d_into(s, strm, gin, part, qhat, err, sb);
        if (lo) bn::launch_add_modes((int)nm, qhat, qlo, strm);
        bn::dft2_inverse_real_into(s, strm, qhat, work, Q_dev);
        if (s->opt.conserve) bn::launch_conserve_on(s, Q_dev, strm);
        e = cudaGetLastError();
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, strm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(strm);
    if (e != cudaSuccess) {
        cudaGetLastError();
        bn::set_last_error(std::string("no-allocation evaluation: ") + cudaGetErrorString(e));
        return BN_ERR_CUDA;
    }
    if (herr != 0) {
        bn::set_last_error("a bounded device wait gave up during the no-allocation evaluation");
        return BN_ERR_TIMEOUT;
    }
    return BN_OK;
}

}  // extern "C"
