// osbf_filter_noalloc: the float32 forward filter without any device allocation.
//
// Some callers cannot call cudaMalloc: real-time pipelines that must not allocate once
// they run (an allocation can synchronise the device and can fail under memory
// pressure), and plug-ins living in a host process whose device memory is owned by
// another allocator.  For them this entry point keeps its scratch -- the two padded
// frames the passes ping-pong between -- in a file-scope device array of fixed size,
// which every GPU that loads the library holds until the process exits.  It launches
// the library's pad and forward kernels with osbf_filter()'s launch plan; it needs no
// context.
#include <cstring>
#include <mutex>

#include "osbf.h"
#include "osbf_internal.h"

namespace {

// Two frames of this many floats each (2 x 16 MiB).
constexpr long long kFrameFloats = OSBF_NOALLOC_MAX_FRAME_FLOATS;

static __device__ __align__(256) float g_noalloc_frames[2 * kFrameFloats];
static __device__ __align__(256) unsigned int g_noalloc_err[64];

// Device addresses of the arrays, looked up once per device (in host code the symbol
// names are only host-side stand-ins and must not be handed to a kernel).
struct DeviceScratch {
    bool ready = false;
    float *frames = nullptr;
    unsigned int *err = nullptr;
    int sms = 0;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

osbf_status setup(int dev, DeviceScratch *&out) {
    if (dev < 0 || dev >= kMaxDevices) return OSBF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScratch &d = g_dev[dev];
    if (!d.ready) {
        void *f = nullptr, *e = nullptr;
        if (cudaGetSymbolAddress(&f, g_noalloc_frames) != cudaSuccess ||
            cudaGetSymbolAddress(&e, g_noalloc_err) != cudaSuccess) {
            cudaGetLastError();
            return OSBF_ECUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return OSBF_ECUDA;
        }
        d.frames = static_cast<float *>(f);
        d.err = static_cast<unsigned int *>(e);
        d.sms = sms;
        d.ready = true;
    }
    out = &d;
    return OSBF_OK;
}

}  // namespace

extern "C" osbf_status osbf_filter_noalloc(const float *in, float *out, int N, int C, int H, int W, int r, int iters,
                                           void *stream) {
    using namespace osbf;
    if (!in || !out || N <= 0 || C <= 0 || H <= 0 || W <= 0 || r < 0 || iters < 0) return OSBF_EINVAL;
    const long long P = (long long)N * C;
    const size_t bytes = sizeof(float) * (size_t)P * H * W;
    if ((const char *)in < (const char *)out + bytes && (const char *)out < (const char *)in + bytes)
        return OSBF_EINVAL;
    if (r > OSBF_MAX_RADIUS) return OSBF_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (r == 0 || iters == 0)
        return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? OSBF_OK : OSBF_ECUDA;

    const int FH = H + 2 * r, FW = W + 2 * r, FWp = (FW + 31) / 32 * 32;
    if (P * FH * (long long)FWp > kFrameFloats) return OSBF_EUNSUPPORTED;  // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OSBF_ECUDA;
    DeviceScratch *d = nullptr;
    osbf_status st = setup(dev, d);
    if (st) return st;
    float *frame[2] = {d->frames, d->frames + kFrameFloats};

    // the error word keeps the last call's value: clear it
    if (cudaMemsetAsync(d->err, 0, sizeof(unsigned int), s) != cudaSuccess) return OSBF_ECUDA;
    if (launch_pad_replicate(Storage::F32, in, frame[0], (int)P, H, W, r, FH, FW, FWp, s) != cudaSuccess)
        return OSBF_ECUDA;
    // one pass per launch, frame to frame, the last pass into the cropped output: the launch
    // plan of osbf_filter(), so both give the same result bit for bit
    int cur = 0;
    for (int pass = 0; pass < iters; ++pass) {
        const bool last = pass == iters - 1;
        GroupLaunch gl;
        gl.st = Storage::F32;
        gl.r = r;
        gl.D = 1;
        gl.src = frame[cur];
        gl.src_pitch = FWp;
        gl.P = (int)P;
        gl.H = H;
        gl.W = W;
        gl.err = d->err;
        gl.sms = d->sms;
        gl.dst = last ? (void *)out : (void *)frame[1 - cur];
        gl.dst_pitch = FWp;
        gl.dst_is_output = last ? 1 : 0;
        const char *what = nullptr;
        if (launch_group(gl, s, &what) != cudaSuccess) return OSBF_ECUDA;
        if (!last) cur = 1 - cur;
    }
    // a bounded tile-load wait that gave up leaves its tile unwritten: read the device error
    // word back (the call returns once the stream has finished the filter)
    unsigned int word = 0;
    if (cudaMemcpyAsync(&word, d->err, sizeof word, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return OSBF_ECUDA;
    if (word) return OSBF_ETIMEOUT;
    return OSBF_OK;
}
