// ecc_tune.cu -- the autotuner: picks tile shapes and histogram
// privatization depth by timing candidates on the device.
//
// Keys: GPU name, SM count, element type and complex.  For each key it
// chooses
//   * the 3D bit-sliced kernel's warps per CTA (4 or 8: warps sharing one
//     shared histogram and one flush), timed in three interleaved rounds on
//     a synthetic 512x512x256 volume, 8 kept unless 4 is at least 3 %
//     faster;
//   * the batched kernel's rows per 2D tile (16, 32, 64) and planes per 3D
//     tile (8, 16, 32), timed on a synthetic uneven batch.
// Results are kept for the process and appended to a text cache
// ($ECC_TUNE_CACHE, else $HOME/.cache/ecc_gb300/tune.txt), so a GPU model is
// tuned once.  ECC_FLAG_NO_AUTOTUNE (or ECC_TUNE=off) keeps the defaults.
#include <cuda_runtime.h>

#include <algorithm>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <sys/stat.h>
#include <vector>

#include "ecc_plan.h"

namespace ecc {
namespace {

// "<key>|3dw" -> {warps per CTA, 0}; "<key>|batch" -> {chunk2d, chunk3d}
struct Choice {
    int a = 0, b = 0;
};

std::mutex g_tune_mu;
std::map<std::string, Choice> g_tuned;
bool g_loaded = false;

std::string cache_path()
{
    if (const char *p = std::getenv("ECC_TUNE_CACHE")) return p;
    const char *home = std::getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/ecc_gb300/tune.txt";
}

void load_cache()
{
    if (g_loaded) return;
    g_loaded = true;
    std::ifstream f(cache_path());
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream is(line);
        std::string key;
        Choice c;
        if (is >> key >> c.a >> c.b) g_tuned[key] = c;
    }
}

void save_choice(const std::string &key, const Choice &c)
{
    const std::string path = cache_path();
    std::string dir = path.substr(0, path.rfind('/'));
    for (size_t i = 1; i <= dir.size(); ++i)
        if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
    std::ofstream f(path, std::ios::app);
    if (f) f << key << ' ' << c.a << ' ' << c.b << '\n';
}

// Smooth-ish synthetic field: a ramp plus blocky hash noise, every value in [lo, hi].
__global__ void synth_fill(unsigned char *d, int64_t n, int esize, int nx, int ny, int lo, int hi)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        unsigned h = (unsigned)((x >> 3) * 73856093u) ^ (unsigned)((y >> 3) * 19349663u) ^ (unsigned)((z >> 3) * 83492791u);
        h ^= h >> 13;
        h *= 0x5bd1e995u;
        const unsigned span = (unsigned)(hi - lo + 1);
        const unsigned v = lo + ((unsigned)(x + y + z) + (h & 63u)) % span;
        if (esize == 1)
            d[i] = (unsigned char)v;
        else
            reinterpret_cast<unsigned short *>(d)[i] = (unsigned short)v;
    }
}

template <class F>
float time_ms(F &&fn, cudaStream_t s, int reps)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    fn();  // warm-up
    cudaEventRecord(a, s);
    for (int r = 0; r < reps; ++r) fn();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return cudaGetLastError() == cudaSuccess ? ms / reps : 1e30f;
}

}  // namespace
}  // namespace ecc

using namespace ecc;

void ecc_plan_s::autotune()
{
    // explicit override (benchmark sweeps): ECC_TILE3D = 4 | 8 warps per CTA
    if (const char *t = std::getenv("ECC_TILE3D")) {
        const int v = std::atoi(t);
        tuned[1] = tuned[3] = v;
    }
    if (d.flags & ECC_FLAG_NO_AUTOTUNE) return;
    if (const char *e = std::getenv("ECC_TUNE"))
        if (!std::strcmp(e, "off")) return;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return;
    std::ostringstream k;
    for (const char *c = prop.name; *c; ++c) k << (*c == ' ' ? '_' : *c);
    k << '|' << num_sms << '|' << (d.dtype == ECC_U16 ? "u16" : "u8") << '|' << d.complex_mode;
    const std::string key = k.str();
    const int key3d = 1 | (d.dtype == ECC_U16 ? 2 : 0);
    const bool want_batch = d.max_images >= 2 && !(d.flags & ECC_FLAG_BATCH_PER_IMAGE);
    bool need3d = true, needb = want_batch;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_cache();
        auto it = g_tuned.find(key + "|3dw");
        if (std::getenv("ECC_TILE3D")) {
            need3d = false;
        } else if (it != g_tuned.end()) {
            tuned[key3d] = it->second.a;
            need3d = false;
        }
        it = g_tuned.find(key + "|batch");
        if (want_batch && it != g_tuned.end()) {
            tuned_batch[0] = it->second.a;
            tuned_batch[1] = it->second.b;
            needb = false;
        }
    }
    if (!need3d && !needb) return;
    const int es = d.dtype == ECC_U16 ? 2 : 1;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    const bool range = !(d.flags & ECC_FLAG_NO_RANGE_CHECK);
    if (need3d) {
        // 3D single-image kernel on a synthetic 512x512x256 volume, with the
        // proportions of large real volumes (how the warps fill the GPU
        // depends on the shape).
        const int nx = 512, ny = 512, nz = 256;
        const int64_t n = (int64_t)nx * ny * nz;
        unsigned char *buf = nullptr;
        Choice c;
        if (cudaMalloc(&buf, n * es) == cudaSuccess) {
            synth_fill<<<1024, 256, 0, s>>>(buf, n, es, nx, ny, d.lo, d.hi);
            Geom g{buf, nz, ny, nx, (int64_t)nx * es, (int64_t)nx * ny * es, 3, es};
            HistDst h{acc, d.lo, nbins};
            // three interleaved rounds, each candidate's best: a single pass
            // in a fixed order is at the mercy of clock ramp-up and noise
            const int cands[2] = {4, 8};
            float best_of[2] = {1e30f, 1e30f};
            for (int round = 0; round < 3; ++round)
                for (int ci = 0; ci < 2; ++ci) {
                    const int tp = cands[ci];
                    const float ms = time_ms(
                        [&] { launch_bitslice(g, 0, nz, h, d.complex_mode, range, status, sched, num_sms, tp, s); },
                        s, 5);
                    best_of[ci] = ms < best_of[ci] ? ms : best_of[ci];
                }
            // 8 warps per CTA unless 4 is at least 3 % faster (8 measured
            // 2-4 % faster at 512^3 uint8, equal at 1024^3 uint16)
            c.a = best_of[0] < 0.97f * best_of[1] ? 4 : 8;
            cudaStreamSynchronize(s);
            cudaFree(buf);
        }
        cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * nbins, s);
        cudaMemsetAsync(status, 0, sizeof(unsigned int), s);
        cudaStreamSynchronize(s);
        cudaGetLastError();
        tuned[key3d] = c.a;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key + "|3dw"] = c;
        save_choice(key + "|3dw", c);
    }
    if (needb) {
        // batched kernel on an uneven synthetic batch (2D and 3D images in one
        // buffer): sides spread over 64-1024 (2D) and 32-252 (3D), enough
        // images to fill the GPU several times over, so the chunk lengths
        // are judged on load balance and halo cost rather than launch
        // latency; the small mix of the first version when the plan cannot
        // hold that many voxels
        std::vector<ecc_image> imgs;
        std::vector<int64_t> offs;
        int64_t total = 0;
        auto make = [&](bool big) {
            imgs.clear();
            offs.clear();
            total = 0;
            const int n2 = big ? std::min(192, d.max_images * 3 / 4 + 1)
                               : (d.max_images >= 48 ? 40 : d.max_images / 2 + 1);
            const int n3 = std::max(0, std::min(big ? 24 : 8, d.max_images - n2));
            for (int i = 0; i < n2 + n3; ++i) {
                ecc_image im{};
                im.dtype = d.dtype;
                if (i < n2) {
                    im.ndim = 2;
                    im.dims[0] = big ? 64 + (97 * i) % 961 : 100 + 37 * i % 400;
                    im.dims[1] = big ? 64 + (61 * i + 300) % 961 : 150 + 53 * i % 500;
                    offs.push_back(total);
                    total += im.dims[0] * im.dims[1];
                } else {
                    const int64_t sd = big ? 32 + 10 * ((7 * (i - n2)) % 23) : 48 + 16 * ((i - n2) % 5);
                    im.ndim = 3;
                    im.dims[0] = im.dims[1] = im.dims[2] = sd;
                    offs.push_back(total);
                    total += sd * sd * sd;
                }
                imgs.push_back(im);
            }
        };
        make(true);
        if (total > d.max_voxels) make(false);
        unsigned char *buf = nullptr;
        long long *out = nullptr;
        Choice c;
        if (total <= d.max_voxels && cudaMalloc(&buf, total * es) == cudaSuccess &&
            cudaMalloc(&out, sizeof(long long) * nbins * imgs.size()) == cudaSuccess) {
            synth_fill<<<1024, 256, 0, s>>>(buf, total, es, 97, 89, d.lo, d.hi);
            for (size_t i = 0; i < imgs.size(); ++i) imgs[i].data = buf + offs[i] * es;
            // candidates: on the 4352-image uneven batch (2D sides 64-1024,
            // 3D sides 32-256) 2D chunks of 64 rows ran 8 % slower than 16
            // or 32, and 3D chunks of 8 or 32 planes 3-5 % slower than 16
            // or 24 (short chunks re-read more halo planes, long ones leave
            // warps idle at the end of the work list).  These lengths serve
            // batches below the work-list kernel's large-batch threshold
            // (which take 32 x 24), so the mix is of that size.  Three
            // interleaved rounds, each candidate's best; the first is kept
            // unless another is at least 3 % faster.
            const int cand[4][2] = {{32, 24}, {32, 16}, {16, 24}, {16, 16}};
            float best_of[4] = {1e30f, 1e30f, 1e30f, 1e30f};
            for (int round = 0; round < 3; ++round)
                for (int ci = 0; ci < 4; ++ci) {
                    release_batch(this);
                    tuned_batch[0] = cand[ci][0];
                    tuned_batch[1] = cand[ci][1];
                    const float ms = time_ms(
                        [&] {
                            ecc_compute_batch(this, (int32_t)imgs.size(), imgs.data(), reinterpret_cast<int64_t *>(out),
                                              s);
                        },
                        s, 3);
                    best_of[ci] = ms < best_of[ci] ? ms : best_of[ci];
                }
            int pick = 0;
            for (int ci = 1; ci < 4; ++ci)
                if (best_of[ci] < 0.97f * best_of[0] && best_of[ci] < best_of[pick]) pick = ci;
            c.a = cand[pick][0];
            c.b = cand[pick][1];
            release_batch(this);
            cudaStreamSynchronize(s);
        }
        if (out) cudaFree(out);
        if (buf) cudaFree(buf);
        cudaMemsetAsync(status, 0, sizeof(unsigned int), s);
        cudaStreamSynchronize(s);
        cudaGetLastError();
        tuned_batch[0] = c.a;
        tuned_batch[1] = c.b;
        if (c.a) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[key + "|batch"] = c;
            save_choice(key + "|batch", c);
        }
    }
    cudaStreamDestroy(s);
}
