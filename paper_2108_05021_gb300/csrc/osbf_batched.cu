// Batched form: many single-plane float32 images of different sizes, radii and pass
// counts in ONE persistent launch, replayed from a CUDA graph cached per job signature.
//
// Work items are (job, pass, tile, kind), listed round by round: every job's pass-0
// tiles, then every job's pass-1 tiles, and so on; after a job's last pass come its crop
// items (kind 1), which copy the frame's interior into the job's output.  CTAs take items
// in that order from a global counter; an item of pass g first waits until all tiles of
// its job's pass g-1 are done (a per-(job, pass) counter).  Every item listed before it
// has already been taken by a resident CTA, so the wait always ends; it is bounded all
// the same (2 s by default, after which the kernel records an error that
// osbf_filter_batched returns as OSBF_ETIMEOUT).
//
// One item is one pass over one tile with the forward's single-pass machinery
// (osbf_fwd2.cuh): the tile's region (tile + r halo) is loaded into shared memory --
// pass 0 from the replicate-padded input by clamped reads, later passes from the job's
// previous frame by coalesced 16-byte L2 loads (another SM wrote it) -- and pass H
// writes its results from registers straight into the job's next frame.  Both loads are
// flat loops over the region's elements.  The sweep code is selected per item by a
// switch on the radius.
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "osbf.h"
#include "osbf_fwd2.cuh"
#include "osbf_internal.h"

osbf_status osbf_ctx_fail(osbf_ctx *ctx, osbf_status code, const char *msg);
void osbf_ctx_count_launches(osbf_ctx *ctx, int n);
void osbf_ctx_reset_launches(osbf_ctx *ctx);
int osbf_ctx_sms(const osbf_ctx *ctx);
int osbf_ctx_device(const osbf_ctx *ctx);
void **osbf_ctx_batch_state(osbf_ctx *ctx);
unsigned long long osbf_ctx_wait_ns(const osbf_ctx *ctx);
osbf_status osbf_forward_run(osbf_ctx *ctx, const void *in, int in_is_frame, int in_pitch, void *out, int out_is_frame,
                             int out_pitch, int P, int H, int W, int r, int iters, osbf_dtype dtype, int depth,
                             int tie, uint8_t *maps, int maps_iter0, long long maps_iter_stride, cudaStream_t s);

namespace osbf {
namespace batched {

constexpr int kMaxR = 8;  // radii served by the persistent launch (larger ones run per job)
constexpr unsigned long long kWaitNs = 2000000000ull;

struct Job {
    const float *in;
    float *out;
    float *frame[2];  // pass g writes frame[g & 1]
    int H, W, FH, FW, FWp, R, iters, tiles_x, ntiles, cnt_base;
    int shift;        // tile k starts at frame column k * TW - shift (TMA boxes start on 16 bytes)
    // The last pass on the output-aligned grid (r % 4 == 0, W % 4 == 0, output on 16 bytes):
    // tile k starts at frame row 32 (k / tiles_x_last) + r and column 128 (k % tiles_x_last)
    // + r, as in a single filter call, whose last pass then shares these tiles' summation
    // order; tiles_x_last x ceil(H / 32) = ntiles_last tiles cover the output.
    int out_grid, tiles_x_last, ntiles_last;
};

// tiles of pass g of a job (the crop, pass `iters`, uses the frame grid)
__device__ __forceinline__ int pass_tiles(const Job &jb, int g) {
    return jb.out_grid && g == jb.iters - 1 ? jb.ntiles_last : jb.ntiles;
}

struct Params {
    unsigned long long wait_ns;  // bound of the dependency wait
    const Job *jobs;
    const int4 *items;           // (job, pass, tile, kind)
    int nitems;
    int *next;                   // item counter
    int *done;                   // tiles finished per (job, pass); the crop is pass `iters`
    unsigned int *err;
    unsigned long long *t_done;  // per job: globaltimer when its last crop tile finished
    unsigned long long *t_start;
};

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The region loads issue kLoadBatch loads per thread before storing any of them: a load
// stored at once into shared memory leaves the thread waiting a full L2 round trip per
// element.
constexpr int kLoadBatch = 16;

// Pass 0's region: the replicate-padded input (clamped reads), zero outside the frame.
// Consecutive threads take consecutive elements of the row-major box.
__device__ void load_padded_input(const Job &jb, const v2::Layout2 &L, float *box, int ty0, int tx0) {
    const int fy0 = ty0 - L.EY, fx0 = tx0 - L.EX;
    const int n = L.RH0 * L.BX;
    for (int e0 = threadIdx.x; e0 < n; e0 += kLoadBatch * v2::NT) {
        float v[kLoadBatch];
#pragma unroll
        for (int i = 0; i < kLoadBatch; ++i) {
            const int e = e0 + i * v2::NT;
            const int y = e / L.BX, x = e - y * L.BX;
            const int fy = fy0 + y, fx = fx0 + x;
            v[i] = 0.f;
            if (e < n && (unsigned)fy < (unsigned)jb.FH && (unsigned)fx < (unsigned)jb.FW)
                v[i] = jb.in[(long long)min(max(fy - jb.R, 0), jb.H - 1) * jb.W + min(max(fx - jb.R, 0), jb.W - 1)];
        }
#pragma unroll
        for (int i = 0; i < kLoadBatch; ++i)
            if (e0 + i * v2::NT < n) box[e0 + i * v2::NT] = v[i];
    }
}

// Later passes' region: the job's previous frame, zero outside it.  The region starts on
// a 16-byte boundary (the tile grid is shifted so that tx0 - r is a multiple of 4), so
// every 4-vector is either wholly left of the frame or starts inside a row; elements past
// the frame's last column are zeroed (the row pitch keeps the vector in bounds).
__device__ void load_frame_region(const Job &jb, const float *src, const v2::Layout2 &L, float *box, int ty0,
                                  int tx0) {
    const int fy0 = ty0 - L.EY, fx0 = tx0 - L.EX;
    const int nv = L.BX / 4;
    const int n = L.RH0 * nv;
    for (int e0 = threadIdx.x; e0 < n; e0 += kLoadBatch * v2::NT) {
        float4 v[kLoadBatch];
#pragma unroll
        for (int i = 0; i < kLoadBatch; ++i) {
            const int e = e0 + i * v2::NT;
            const int y = e / nv, x = (e - y * nv) * 4;
            const int fy = fy0 + y, fx = fx0 + x;
            v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < n && (unsigned)fy < (unsigned)jb.FH && fx >= 0 && fx < jb.FW) {
                v[i] = __ldcg(reinterpret_cast<const float4 *>(src + (long long)fy * jb.FWp + fx));
                if (fx + 1 >= jb.FW) v[i].y = 0.f;
                if (fx + 2 >= jb.FW) v[i].z = 0.f;
                if (fx + 3 >= jb.FW) v[i].w = 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < kLoadBatch; ++i) {
            const int e = e0 + i * v2::NT;
            if (e < n) {
                const int y = e / nv, x = (e - y * nv) * 4;
                *reinterpret_cast<float4 *>(box + y * L.BX + x) = v[i];
            }
        }
    }
}

// One pass over one tile.
template <int R>
__device__ void process(const Job &jb, int g, int tile, unsigned char *smem) {
    const v2::Layout2 L = v2::make_layout2<float>(R, 1, true);
    float *box = reinterpret_cast<float *>(smem + L.off_in);
    float *A = reinterpret_cast<float *>(smem + L.off_ab);
    const bool og = jb.out_grid && g == jb.iters - 1;
    const int ty0 = og ? (tile / jb.tiles_x_last) * v2::TH + R : (tile / jb.tiles_x) * v2::TH;
    const int tx0 = og ? (tile % jb.tiles_x_last) * v2::TW + R : (tile % jb.tiles_x) * v2::TW - jb.shift;
    if (g == 0)
        load_padded_input(jb, L, box, ty0, tx0);
    else
        load_frame_region(jb, jb.frame[(g - 1) & 1], L, box, ty0, tx0);
    __syncthreads();
    v2::pass_v2<R, v2::TH + 2 * R>(box, L.BX, A, L.P2, L.RH0, L.RW0);
    __syncthreads();
    v2::Geom2 gm;
    gm.RHo = v2::TH;
    gm.RWo = v2::TW;
    gm.fy0 = ty0;
    gm.fx0 = tx0;
    gm.FH = jb.FH;
    gm.FW = jb.FW;
    gm.iy0 = 0;
    gm.iy1 = v2::TH;
    gm.ix0 = 0;
    gm.ix1 = v2::TW;
    gm.oy = gm.ox = 0;
    gm.ly = jb.FH;
    gm.lx = jb.FW;
    gm.MP = 0;
    v2::pass_h2<R, float, false, false, true>(box, L.BX, R, A, L.P2, nullptr, 0, jb.frame[g & 1], jb.FWp, gm,
                                              nullptr);
}

// The crop: the interior of the last frame into the job's output (coalesced rows).
__device__ void crop(const Job &jb, int tile) {
    const int ty0 = (tile / jb.tiles_x) * v2::TH;
    const int tx0 = (tile % jb.tiles_x) * v2::TW - jb.shift;
    const float *src = jb.frame[(jb.iters - 1) & 1];
    for (int i = threadIdx.x; i < v2::TH * v2::TW; i += v2::NT) {
        const int fy = ty0 + i / v2::TW, fx = tx0 + i % v2::TW;
        const int oy = fy - jb.R, ox = fx - jb.R;
        if ((unsigned)oy < (unsigned)jb.H && (unsigned)ox < (unsigned)jb.W)
            jb.out[(long long)oy * jb.W + ox] = __ldcg(src + (long long)fy * jb.FWp + fx);
    }
}

// L2 prefetch of the rows an item will read (a tile's region of the previous frame, of the
// clamped input for pass 0, or a crop tile's frame rows), one instruction per 128-byte
// line, spread over the CTA.  The frames of a whole batch do not stay in L2 between pass
// rounds, so without it every region load waits on DRAM.
__device__ __forceinline__ void prefetch_rows(const float *base, long long pitch, int y0, int y1, int x0, int x1) {
    if (y0 >= y1 || x0 >= x1) return;
    const int l0 = x0 >> 5, l1 = (x1 - 1) >> 5;  // 32 floats per 128-byte line
    const int nl = l1 - l0 + 1, n = (y1 - y0) * nl;
    for (int e = threadIdx.x; e < n; e += v2::NT) {
        const int y = y0 + e / nl, l = l0 + e % nl;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (long long)y * pitch + (long long)l * 32));
    }
}

__device__ void prefetch_item(const Job &jb, int g, int tile, int crop_item) {
    if (crop_item) {
        const int ty0 = (tile / jb.tiles_x) * v2::TH, tx0 = (tile % jb.tiles_x) * v2::TW - jb.shift;
        prefetch_rows(jb.frame[(jb.iters - 1) & 1], jb.FWp, max(ty0, jb.R), min(ty0 + v2::TH, jb.R + jb.H),
                      max(tx0, jb.R), min(tx0 + v2::TW, jb.R + jb.W));
        return;
    }
    const v2::Layout2 L = v2::make_layout2<float>(jb.R, 1, true);
    const bool og = jb.out_grid && g == jb.iters - 1;
    const int ty0 = og ? (tile / jb.tiles_x_last) * v2::TH + jb.R : (tile / jb.tiles_x) * v2::TH;
    const int tx0 = og ? (tile % jb.tiles_x_last) * v2::TW + jb.R : (tile % jb.tiles_x) * v2::TW - jb.shift;
    const int fy0 = ty0 - L.EY, fx0 = tx0 - L.EX;
    if (g == 0)  // the region's frame rows and columns, clamped into the unpadded input
        prefetch_rows(jb.in, jb.W, max(fy0 - jb.R, 0), min(fy0 + L.RH0 - jb.R, jb.H), max(fx0 - jb.R, 0),
                      min(fx0 + L.BX - jb.R, jb.W));
    else
        prefetch_rows(jb.frame[(g - 1) & 1], jb.FWp, max(fy0, 0), min(fy0 + L.RH0, jb.FH), max(fx0, 0),
                      min(fx0 + L.BX, jb.FW));
}

__global__ void __launch_bounds__(v2::NT) osbf_batched_kernel(const Params p) {
    extern __shared__ __align__(128) unsigned char bsmem[];
    __shared__ int s_item, s_next;
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        atomicMin(p.t_start, now_ns());
        s_fail = 0;
        s_item = atomicAdd(p.next, 1);
    }
    for (;;) {
        __syncthreads();
        const int item = s_item;
        if (item >= p.nitems) break;
        // the item after this one is taken now, so its rows can be prefetched during this one
        if (threadIdx.x == 0) s_next = atomicAdd(p.next, 1);
        const int4 it = p.items[item];
        const Job jb = p.jobs[it.x];
        const int g = it.y;
        if (threadIdx.x == 0 && g > 0) {
            // the job's previous pass must be complete (bounded wait)
            const volatile int *cnt = p.done + jb.cnt_base + g - 1;
            const unsigned long long t0 = now_ns();
            const int need = pass_tiles(jb, g - 1);
            while (*cnt < need) {
                if (now_ns() - t0 > p.wait_ns) {
                    atomicOr(p.err, 1u);
                    s_fail = 1;
                    break;
                }
                __nanosleep(128);
            }
            __threadfence();
        }
        __syncthreads();
        if (s_fail) break;
        {
            const int nx = s_next;
            if (nx < p.nitems) {
                const int4 it2 = p.items[nx];
                prefetch_item(p.jobs[it2.x], it2.y, it2.z, it2.w);
            }
        }
        if (it.w) {
            crop(jb, it.z);
        } else {
            switch (jb.R) {
            case 1: process<1>(jb, g, it.z, bsmem); break;
            case 2: process<2>(jb, g, it.z, bsmem); break;
            case 3: process<3>(jb, g, it.z, bsmem); break;
            case 4: process<4>(jb, g, it.z, bsmem); break;
            case 5: process<5>(jb, g, it.z, bsmem); break;
            case 6: process<6>(jb, g, it.z, bsmem); break;
            case 7: process<7>(jb, g, it.z, bsmem); break;
            default: process<8>(jb, g, it.z, bsmem); break;
            }
        }
        // every thread's stores of this tile precede the barrier; thread 0's fence, which
        // is cumulative over them, publishes them before the tile is counted
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const int prev = atomicAdd(p.done + jb.cnt_base + g, 1);
            if (it.w && prev + 1 == jb.ntiles) p.t_done[it.x] = now_ns();
            s_item = s_next;
        }
    }
}

}  // namespace batched
}  // namespace osbf

using namespace osbf;

namespace {

struct Planned {
    cudaGraphExec_t exec = nullptr;
    char *arena = nullptr;
    unsigned int *err = nullptr;
    unsigned long long *t_done = nullptr, *t_start = nullptr;
    int njobs = 0;
};

// How a batch is laid out and launched: the job order within each pass round (0: as given,
// 1: by decreasing work, H x W x passes, so the longest chains start first; 2: grouped by
// radius, then by decreasing work -- CTAs that run at the same time then run the same
// radius's unrolled sweep, which keeps one variant's code in the instruction cache) and the
// resident CTAs per SM.  osbf_autotune_batched() times the candidates on the batch itself.
struct Policy {
    int order = 2;  // untuned: grouped by radius
    int ctas_per_sm = 0;  // 0: as many as fit
};

struct BatchState {
    std::map<std::vector<long long>, Planned> plans;  // job signature + policy -> graph and arena
    std::map<std::vector<long long>, Policy> tuned;   // job signature -> tuned policy
    const Planned *last = nullptr;                    // for osbf_batched_latencies()
};

BatchState *state(osbf_ctx *ctx) {
    void **slot = osbf_ctx_batch_state(ctx);
    if (!*slot) *slot = new BatchState();
    return (BatchState *)*slot;
}

}  // namespace

void osbf_batched_free(osbf_ctx *ctx) {
    void **slot = osbf_ctx_batch_state(ctx);
    if (!*slot) return;
    BatchState *st = (BatchState *)*slot;
    for (auto &kv : st->plans) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaFree(kv.second.arena);
    }
    delete st;
    *slot = nullptr;
}

bool osbf_ctx_tuned_elsewhere(osbf_ctx *ctx, int r, long long pixels);

namespace {

// Jobs the persistent launch takes: 1 <= r <= 8, iters >= 1, and no tuned single-call
// choice of another kernel or depth (those run as plain filter calls).
bool persistent_job(osbf_ctx *ctx, const osbf_job &q) {
    return q.r >= 1 && q.iters >= 1 && q.r <= batched::kMaxR &&
           !osbf_ctx_tuned_elsewhere(ctx, q.r, (long long)q.H * q.W);
}

// The job signature: the batch size, the wait bound and every persistent job's pointers,
// sizes, radius and pass count (the key of the cached graphs and of the tuned policies).
std::vector<long long> job_signature(osbf_ctx *ctx, const osbf_job *jobs, int njobs) {
    std::vector<long long> sig;
    sig.push_back(njobs);
    sig.push_back((long long)osbf_ctx_wait_ns(ctx));
    for (int j = 0; j < njobs; ++j) {
        const osbf_job &q = jobs[j];
        if (persistent_job(ctx, q))
            sig.insert(sig.end(), {(long long)(uintptr_t)q.in, (long long)(uintptr_t)q.out, q.H, q.W, q.r, q.iters});
    }
    return sig;
}

// The batched call with a given policy (force), or with the tuned one (force == nullptr).
osbf_status batched_run(osbf_ctx *ctx, const osbf_job *jobs, int njobs, void *stream, const Policy *force) {
    if (!ctx) return OSBF_EINVAL;
    osbf_ctx_reset_launches(ctx);
    if (njobs < 0 || (njobs > 0 && !jobs)) return osbf_ctx_fail(ctx, OSBF_EINVAL, "bad job list");
    cudaStream_t s = (cudaStream_t)stream;
    for (int j = 0; j < njobs; ++j) {
        const osbf_job &q = jobs[j];
        if (!q.in || !q.out || q.H <= 0 || q.W <= 0 || q.r < 0 || q.iters < 0)
            return osbf_ctx_fail(ctx, OSBF_EINVAL, "bad job");
        if (q.r > OSBF_MAX_RADIUS) return osbf_ctx_fail(ctx, OSBF_EUNSUPPORTED, "job radius exceeds OSBF_MAX_RADIUS");
        if (q.in == q.out) return osbf_ctx_fail(ctx, OSBF_EINVAL, "job in and out alias");
    }
    BatchState *bs = state(ctx);

    // the persistent launch takes jobs with 1 <= r <= 8 and iters >= 1; the rest run alone
    std::vector<int> pj;
    std::vector<long long> sig = job_signature(ctx, jobs, njobs);
    for (int j = 0; j < njobs; ++j) {
        const osbf_job &q = jobs[j];
        if (q.r == 0 || q.iters == 0) {
            if (cudaMemcpyAsync(q.out, q.in, sizeof(float) * (size_t)q.H * q.W, cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess)
                return osbf_ctx_fail(ctx, OSBF_ECUDA, "copy failed");
        } else if (!persistent_job(ctx, q)) {
            // radii beyond the persistent kernel's, and jobs whose tuned forward is another
            // kernel or depth: a plain filter call each (which applies the tuned choice)
            osbf_status e = osbf_forward_run(ctx, q.in, 0, 0, q.out, 0, 0, 1, q.H, q.W, q.r, q.iters, OSBF_F32, 0, 0,
                                             nullptr, 0, 0, s);
            if (e) return e;
        } else {
            pj.push_back(j);
        }
    }
    if (pj.empty()) return OSBF_OK;

    Policy pol;
    if (force) {
        pol = *force;
    } else {
        auto tit = bs->tuned.find(sig);
        if (tit != bs->tuned.end()) pol = tit->second;
    }
    sig.push_back(pol.order);
    sig.push_back(pol.ctas_per_sm);
    auto git = bs->plans.find(sig);
    if (git == bs->plans.end()) {
        // ---- plan: jobs, items in round order, counters, arena ----
        std::vector<batched::Job> hj(pj.size());
        size_t frame_floats = 0;
        int cnt = 0, max_iters = 0;
        size_t smem = 0;
        for (size_t k = 0; k < pj.size(); ++k) {
            const osbf_job &q = jobs[pj[k]];
            batched::Job &b = hj[k];
            b.in = q.in;
            b.out = q.out;
            b.H = q.H;
            b.W = q.W;
            b.R = q.r;
            b.FH = q.H + 2 * q.r;
            b.FW = q.W + 2 * q.r;
            b.FWp = (b.FW + 31) / 32 * 32;
            b.iters = q.iters;
            b.shift = (4 - q.r % 4) % 4;
            b.tiles_x = (b.FW - 1 + b.shift) / v2::TW + 1;
            b.ntiles = b.tiles_x * ((b.FH + v2::TH - 1) / v2::TH);
            // the single-call plan's condition for the output-aligned last pass
            b.out_grid = q.r % 4 == 0 && q.W % 4 == 0 && ((uintptr_t)q.out & 15) == 0;
            b.tiles_x_last = (q.W + v2::TW - 1) / v2::TW;
            b.ntiles_last = b.tiles_x_last * ((q.H + v2::TH - 1) / v2::TH);
            b.cnt_base = cnt;
            cnt += b.iters + 1;  // the passes, then the crop
            max_iters = std::max(max_iters, b.iters);
            frame_floats += 2 * (size_t)b.FH * b.FWp;
            smem = std::max(smem, (size_t)v2::make_layout2<float>(q.r, 1, true).bytes);
        }
        std::vector<size_t> korder(hj.size());
        for (size_t k = 0; k < hj.size(); ++k) korder[k] = k;
        if (pol.order == 1 || pol.order == 2)
            std::stable_sort(korder.begin(), korder.end(), [&](size_t a, size_t b) {
                if (pol.order == 2 && hj[a].R != hj[b].R) return hj[a].R < hj[b].R;
                return (long long)hj[a].H * hj[a].W * hj[a].iters > (long long)hj[b].H * hj[b].W * hj[b].iters;
            });
        std::vector<int4> items;
        for (int g = 0; g <= max_iters; ++g)
            for (size_t k : korder)
                if (g <= hj[k].iters)
                    for (int t = 0; t < (hj[k].out_grid && g == hj[k].iters - 1 ? hj[k].ntiles_last : hj[k].ntiles); ++t)
                        items.push_back(make_int4((int)k, g, t, g == hj[k].iters));
        // arena: jobs | items | next | counters | err | t_done | t_start | frames
        size_t off = 0;
        auto take = [&](size_t bytes) {
            const size_t o = off;
            off += (bytes + 255) & ~(size_t)255;
            return o;
        };
        const size_t o_jobs = take(sizeof(batched::Job) * hj.size());
        const size_t o_items = take(sizeof(int4) * items.size());
        const size_t o_next = take(sizeof(int));
        const size_t o_done = take(sizeof(int) * (size_t)cnt);
        const size_t o_err = take(sizeof(unsigned int));
        const size_t o_tdone = take(sizeof(unsigned long long) * hj.size());
        const size_t o_tstart = take(sizeof(unsigned long long));
        const size_t o_frames = take(sizeof(float) * frame_floats);
        char *arena = nullptr;
        if (cudaMalloc(&arena, off) != cudaSuccess) {
            cudaGetLastError();
            return osbf_ctx_fail(ctx, OSBF_ENOMEM, "batched arena allocation failed");
        }
        float *fr = (float *)(arena + o_frames);
        for (auto &b : hj)
            for (int f = 0; f < 2; ++f) {
                b.frame[f] = fr;
                fr += (size_t)b.FH * b.FWp;
            }
        if (cudaMemcpy(arena + o_jobs, hj.data(), sizeof(batched::Job) * hj.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(arena + o_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            cudaFree(arena);
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "batched plan upload failed");
        }
        batched::Params p;
        p.wait_ns = osbf_ctx_wait_ns(ctx);
        if (p.wait_ns == 0) p.wait_ns = batched::kWaitNs;
        p.jobs = (const batched::Job *)(arena + o_jobs);
        p.items = (const int4 *)(arena + o_items);
        p.nitems = (int)items.size();
        p.next = (int *)(arena + o_next);
        p.done = (int *)(arena + o_done);
        p.err = (unsigned int *)(arena + o_err);
        p.t_done = (unsigned long long *)(arena + o_tdone);
        p.t_start = (unsigned long long *)(arena + o_tstart);
        if (cudaFuncSetAttribute(batched::osbf_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess) {
            cudaFree(arena);
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "shared memory attribute");
        }
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched::osbf_batched_kernel, v2::NT, smem);
        if (occ < 1) occ = 1;
        if (pol.ctas_per_sm > 0 && pol.ctas_per_sm < occ) occ = pol.ctas_per_sm;
        int grid = occ * osbf_ctx_sms(ctx);  // all CTAs resident: every wait is on a running CTA
        if (grid > (int)items.size()) grid = (int)items.size();

        // ---- capture: reset the counters, then the persistent launch ----
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            cudaFree(arena);
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "stream creation failed");
        }
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemsetAsync(arena + o_next, 0, o_tstart - o_next, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(arena + o_tstart, 0xff, sizeof(unsigned long long), cs);
        if (e == cudaSuccess) {
            batched::osbf_batched_kernel<<<grid, v2::NT, smem, cs>>>(p);
            e = cudaGetLastError();
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e2 == cudaSuccess) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            cudaFree(arena);
            return osbf_ctx_fail(ctx, OSBF_ECUDA, cudaGetErrorString(e));
        }
        Planned pl;
        pl.exec = exec;
        pl.arena = arena;
        pl.err = p.err;
        pl.t_done = p.t_done;
        pl.t_start = p.t_start;
        pl.njobs = (int)hj.size();
        git = bs->plans.emplace(sig, pl).first;
    }
    const Planned &pl = git->second;
    bs->last = &pl;
    cudaError_t e = cudaGraphLaunch(pl.exec, s);
    if (e != cudaSuccess) return osbf_ctx_fail(ctx, OSBF_ECUDA, cudaGetErrorString(e));
    osbf_ctx_count_launches(ctx, 1);
    // the bounded waits report through the arena's error word
    unsigned int w = 0;
    if (cudaMemcpyAsync(&w, pl.err, sizeof w, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return osbf_ctx_fail(ctx, OSBF_ECUDA, "batched launch failed");
    if (w) return osbf_ctx_fail(ctx, OSBF_ETIMEOUT, "a batched item waited too long for its previous pass");
    return OSBF_OK;
}

}  // namespace

extern "C" {

osbf_status osbf_filter_batched(osbf_ctx *ctx, const osbf_job *jobs, int njobs, void *stream) {
    return batched_run(ctx, jobs, njobs, stream, nullptr);
}

osbf_status osbf_autotune_batched(osbf_ctx *ctx, const osbf_job *jobs, int njobs, void *stream) {
    if (!ctx) return OSBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int occ = 0;
    {
        size_t smem = 0;
        for (int j = 0; j < njobs; ++j)
            if (jobs && persistent_job(ctx, jobs[j]))
                smem = std::max(smem, (size_t)v2::make_layout2<float>(jobs[j].r, 1, true).bytes);
        if (smem == 0) return batched_run(ctx, jobs, njobs, stream, nullptr);  // nothing to tune
        if (cudaFuncSetAttribute(batched::osbf_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched::osbf_batched_kernel, v2::NT, smem) !=
                cudaSuccess)
            return osbf_ctx_fail(ctx, OSBF_ECUDA, "occupancy query failed");
        if (occ < 1) occ = 1;
    }
    std::vector<Policy> cand;
    for (int order = 0; order < 3; ++order)
        for (int c = occ; c >= 1 && c >= occ - 1; --c) {
            Policy p;
            p.order = order;
            p.ctas_per_sm = c;
            cand.push_back(p);
        }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Policy best = cand[0];
    float best_ms = 1e30f;
    osbf_status st = OSBF_OK;
    for (const Policy &p : cand) {
        st = batched_run(ctx, jobs, njobs, stream, &p);  // builds and caches this policy's graph
        if (st) break;
        cudaEventRecord(e0, s);
        for (int k = 0; k < 3 && !st; ++k) st = batched_run(ctx, jobs, njobs, stream, &p);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = p;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    // record it under the job signature (the same key osbf_filter_batched() looks up)
    BatchState *bs = state(ctx);
    const std::vector<long long> sig = job_signature(ctx, jobs, njobs);
    bs->tuned[sig] = best;
    return OSBF_OK;
}

int osbf_batched_policy(osbf_ctx *ctx, const osbf_job *jobs, int njobs, int *order, int *ctas_per_sm) {
    if (!ctx || !order || !ctas_per_sm) return 0;
    BatchState *bs = state(ctx);
    const std::vector<long long> sig = job_signature(ctx, jobs, njobs);
    auto it = bs->tuned.find(sig);
    if (it == bs->tuned.end()) {
        *order = Policy().order;
        *ctas_per_sm = 0;
        return 0;
    }
    *order = it->second.order;
    *ctas_per_sm = it->second.ctas_per_sm;
    return 1;
}

// Per-image latency of the last osbf_filter_batched() call on `ctx` (see osbf.h).
int osbf_batched_latencies(osbf_ctx *ctx, unsigned long long *ns, int cap) {
    if (!ctx || !ns || cap <= 0) return 0;
    BatchState *bs = state(ctx);
    const Planned *pl = bs->last;
    if (!pl || pl->njobs == 0) return 0;
    std::vector<unsigned long long> t(pl->njobs);
    unsigned long long t0 = 0;
    if (cudaMemcpy(t.data(), pl->t_done, sizeof(unsigned long long) * pl->njobs, cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(&t0, pl->t_start, sizeof t0, cudaMemcpyDeviceToHost) != cudaSuccess)
        return 0;
    const int n = pl->njobs < cap ? pl->njobs : cap;
    for (int i = 0; i < n; ++i) ns[i] = t[i] > t0 ? t[i] - t0 : 0;
    return n;
}

}  // extern "C"
