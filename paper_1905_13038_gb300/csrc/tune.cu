// Autotuner: launch parameters measured on the device and kept in a JSON
// cache that persists across runs.
//
// What is tuned (the arithmetic and therefore every output bit are the same
// for every candidate; only the work split changes):
//   window   tile height, edge-tile fraction and stripe pre-pass of the
//            Sauvola / Niblack window kernel (binarize precisions);
//   quantile row-band height of the local-quantile kernel;
//   batch    tile rows of the batched window and quantile kernels, as
//            multiples of each job's window height.
// Candidates are timed with CUDA events on the caller's stream (one
// untimed run, then the median of several, each after reading a buffer
// larger than L2 so that the input comes from HBM as it does for a stream of
// distinct images; with three runs and their mean, run-to-run spread of the
// window kernel (~2 %) was as large as the gap between the best candidates
// and a slower tile schedule could win), the fastest is stored under a key of
// GPU name and SM count, kernel, precision (or quantile class), window-size
// buckets (next power of two of h and w) and image-size bucket (half octaves
// of H x W), and the cache is written back to its file.
//
// BZ_TUNE: unset = use cached entries, never tune implicitly; 0 = ignore the
// cache (built-in heuristics only); 1 = tune on a cache miss inside the call
// (synchronous).  The explicit bz_autotune_* calls always tune.  The cache
// file is BZ_TUNE_CACHE, else $XDG_CACHE_HOME/paper_1905_13038_gb300/
// tune.json, else $HOME/.cache/paper_1905_13038_gb300/tune.json.  A missing
// or unreadable file is an empty cache; it is rewritten whole (temporary file
// and rename) after each tuning.
#include <algorithm>
#include <errno.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "batch_internal.h"
#include "bz_internal.h"

namespace bz {

// ------------------------------------------------------------ the cache --
static std::mutex g_tune_mu;
static std::map<std::string, TuneCfg> g_tune;
static bool g_tune_loaded = false;
static std::string g_tune_path;

static thread_local const TuneCfg *tl_override = nullptr;
static thread_local bool tl_force = false;

const TuneCfg *tune_override() { return tl_override; }
bool tune_forced() { return tl_force; }
TuneForce::TuneForce() : prev_(tl_force) { tl_force = true; }
TuneForce::~TuneForce() { tl_force = prev_; }

// Whether a launch tunes now: forced by an explicit bz_autotune_* call, or
// BZ_TUNE=1 and no cached entry.
bool tune_now(bool have) { return tl_force || (!have && tune_env() == 1); }

TuneScope::TuneScope(const TuneCfg *c) : prev_(tl_override) { tl_override = c; }
TuneScope::~TuneScope() { tl_override = prev_; }

int tune_env()
{
    static const int v = [] {
        const char *e = getenv("BZ_TUNE");
        return e ? (atoi(e) != 0 ? 1 : 0) : -1;
    }();
    return v;
}

static std::string default_cache_path()
{
    const char *p = getenv("BZ_TUNE_CACHE");
    if (p && *p)
        return p;
    const char *x = getenv("XDG_CACHE_HOME");
    if (x && *x)
        return std::string(x) + "/paper_1905_13038_gb300/tune.json";
    const char *h = getenv("HOME");
    return std::string(h && *h ? h : ".") + "/.cache/paper_1905_13038_gb300/tune.json";
}

int dim_bucket(int v)
{
    int b = 1;
    while (b < v && b < (1 << 30))
        b <<= 1;
    return b;
}

int size_bucket(int64_t H, int64_t W)
{
    const double px = (double)H * (double)W;
    return px < 1.0 ? 0 : (int)floor(2.0 * log2(px));
}

std::string tune_key(const char *gpu, const char *kernel, int cls, int h, int w, int64_t H, int64_t W)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%s|%d|h%d|w%d|s%d", gpu, kernel, cls, dim_bucket(h), dim_bucket(w),
             size_bucket(H, W));
    return buf;
}

// "<name>/<SMs>" of the current device (cached per device).
std::string device_tag()
{
    static std::mutex mu;
    static std::string tags[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return "nodevice";
    }
    std::lock_guard<std::mutex> lk(mu);
    if (tags[dev].empty()) {
        cudaDeviceProp p;
        if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
            cudaGetLastError();
            return "nodevice";
        }
        tags[dev] = std::string(p.name) + "/" + std::to_string(p.multiProcessorCount);
    }
    return tags[dev];
}

// --- a small reader for the cache's own JSON layout:
// {"version": 1, "entries": {"<key>": {"tile_h": n, "edge": x, "stripes": n,
//  "us": x}, ...}}
namespace {
struct Reader {
    const char *p, *end;
    void ws()
    {
        while (p < end && (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t'))
            p++;
    }
    bool lit(char c)
    {
        ws();
        if (p < end && *p == c) {
            p++;
            return true;
        }
        return false;
    }
    bool str(std::string &s)
    {
        ws();
        if (p >= end || *p != '"')
            return false;
        p++;
        s.clear();
        while (p < end && *p != '"') {
            if (*p == '\\' || (unsigned char)*p < 0x20)
                return false;  // keys never need escapes
            s.push_back(*p++);
        }
        if (p >= end)
            return false;
        p++;
        return true;
    }
    bool num(double &v)
    {
        ws();
        char *q = nullptr;
        errno = 0;
        v = strtod(p, &q);
        if (q == p || errno != 0 || q > end || !isfinite(v))
            return false;
        p = q;
        return true;
    }
};

bool parse_cache(const std::string &text, std::map<std::string, TuneCfg> &out)
{
    Reader r{text.data(), text.data() + text.size()};
    std::map<std::string, TuneCfg> m;
    if (!r.lit('{'))
        return false;
    bool have_entries = false;
    bool first = true;
    while (!r.lit('}')) {
        if (!first && !r.lit(','))
            return false;
        first = false;
        std::string name;
        if (!r.str(name) || !r.lit(':'))
            return false;
        if (name == "version") {
            double v;
            if (!r.num(v) || v != 1.0)
                return false;
        } else if (name == "entries") {
            if (!r.lit('{'))
                return false;
            bool f2 = true;
            while (!r.lit('}')) {
                if (!f2 && !r.lit(','))
                    return false;
                f2 = false;
                std::string key;
                if (!r.str(key) || !r.lit(':') || !r.lit('{'))
                    return false;
                TuneCfg c;
                int seen = 0;
                bool f3 = true;
                while (!r.lit('}')) {
                    if (!f3 && !r.lit(','))
                        return false;
                    f3 = false;
                    std::string field;
                    double v;
                    if (!r.str(field) || !r.lit(':') || !r.num(v))
                        return false;
                    if (field == "tile_h") {
                        c.tile_h = (int32_t)v;
                        seen |= 1;
                    } else if (field == "edge") {
                        c.edge = (float)v;
                        seen |= 2;
                    } else if (field == "stripes") {
                        c.stripes = (int32_t)v;
                        seen |= 4;
                    } else if (field == "us") {
                        c.us = (float)v;
                        seen |= 8;
                    } else {
                        return false;
                    }
                }
                if (seen != 15 || c.tile_h < 0 || c.tile_h > (1 << 30) || c.edge < 0.0f || c.edge > 1.0f ||
                    c.stripes < -1 || c.stripes > 64)
                    return false;
                m[key] = c;
            }
            have_entries = true;
        } else {
            return false;
        }
    }
    r.ws();
    if (r.p != r.end || !have_entries)
        return false;
    out.swap(m);
    return true;
}

std::string format_cache(const std::map<std::string, TuneCfg> &m)
{
    std::string s = "{\"version\": 1, \"entries\": {";
    bool first = true;
    for (const auto &kv : m) {
        char buf[512];
        snprintf(buf, sizeof buf, "%s\n  \"%s\": {\"tile_h\": %d, \"edge\": %.4f, \"stripes\": %d, \"us\": %.3f}",
                 first ? "" : ",", kv.first.c_str(), kv.second.tile_h, kv.second.edge, kv.second.stripes,
                 kv.second.us);
        s += buf;
        first = false;
    }
    s += "\n}}\n";
    return s;
}

bool read_file(const std::string &path, std::string &text)
{
    FILE *f = fopen(path.c_str(), "rb");
    if (!f)
        return false;
    char buf[4096];
    size_t n;
    text.clear();
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) {
        text.append(buf, n);
        if (text.size() > (16u << 20)) {  // not a cache of this library
            fclose(f);
            return false;
        }
    }
    fclose(f);
    return true;
}

void make_parent_dirs(const std::string &path)
{
    for (size_t i = 1; i < path.size(); i++)
        if (path[i] == '/')
            mkdir(path.substr(0, i).c_str(), 0755);
}
}  // namespace

// Both with g_tune_mu held.
static void load_locked()
{
    if (g_tune_loaded)
        return;
    g_tune_loaded = true;
    if (g_tune_path.empty())
        g_tune_path = default_cache_path();
    std::string text;
    std::map<std::string, TuneCfg> m;
    if (read_file(g_tune_path, text) && parse_cache(text, m))
        g_tune.swap(m);
}

static bool save_locked(const std::string &path)
{
    make_parent_dirs(path);
    const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f)
        return false;
    const std::string s = format_cache(g_tune);
    const bool ok = fwrite(s.data(), 1, s.size(), f) == s.size();
    if (fclose(f) != 0 || !ok || rename(tmp.c_str(), path.c_str()) != 0) {
        remove(tmp.c_str());
        return false;
    }
    return true;
}

bool tune_get(const std::string &key, TuneCfg &c)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_locked();
    const auto it = g_tune.find(key);
    if (it == g_tune.end())
        return false;
    c = it->second;
    return true;
}

void tune_put(const std::string &key, const TuneCfg &c, bool save)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_locked();
    g_tune[key] = c;
    if (save)
        save_locked(g_tune_path);
}

// --------------------------------------------------------- the searches --
// A device buffer larger than L2, read before each timed run (k_l2_evict) so
// that a candidate is timed with its input coming from HBM and with L2
// holding clean lines, as in a stream of distinct images (null when it
// cannot be had: the runs are then timed warm).  One per device, allocated
// and zeroed by the first tuning call on it.
__global__ void k_l2_evict(const uint4 *p, size_t n, unsigned *sink)
{
    uint32_t acc = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 v = __ldcg(p + i);
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9E3779B9u)  // never for the zeroed buffer; keeps the loads
        atomicAdd(sink, 1u);
}

static void *l2_flush_buffer(size_t &bytes)
{
    static std::mutex mu;
    static void *bufs[64] = {nullptr};
    static size_t sizes[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!bufs[dev]) {
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        const size_t want = (size_t)(l2 > 0 ? l2 : (128 << 20)) * 5 / 4;
        if (cudaMalloc(&bufs[dev], want + 256) != cudaSuccess) {
            cudaGetLastError();
            bufs[dev] = nullptr;
            return nullptr;
        }
        if (cudaMemset(bufs[dev], 0, want + 256) != cudaSuccess) {
            cudaFree(bufs[dev]);
            cudaGetLastError();
            bufs[dev] = nullptr;
            return nullptr;
        }
        sizes[dev] = want;
    }
    bytes = sizes[dev];
    return bufs[dev];
}

// Median device time of `launch` (a callable returning cudaError_t) on
// `stream`: one untimed run, then `reps` (at most 15) timed ones, each after
// an L2 flush.  Negative on error.
template <typename F>
static double time_on(cudaStream_t stream, int reps, F &&launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a)
            cudaEventDestroy(a);
        cudaGetLastError();
        return -1.0;
    }
    size_t fbytes = 0;
    void *fbuf = l2_flush_buffer(fbytes);
    float ts[15];
    reps = reps < 1 ? 1 : (reps > 15 ? 15 : reps);
    bool ok = launch() == cudaSuccess;
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int r = 0; r < reps && ok; r++) {
        if (fbuf) {
            k_l2_evict<<<sms * 4, 256, 0, stream>>>((const uint4 *)fbuf, fbytes / 16,
                                                    (unsigned *)((char *)fbuf + fbytes));
            ok = cudaGetLastError() == cudaSuccess;
        }
        float t = 0.0f;
        ok = ok && cudaEventRecord(a, stream) == cudaSuccess && launch() == cudaSuccess &&
             cudaEventRecord(b, stream) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
             cudaEventElapsedTime(&t, a, b) == cudaSuccess;
        ts[r] = t;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaGetLastError();
    if (!ok)
        return -1.0;
    std::sort(ts, ts + reps);
    return reps % 2 ? ts[reps / 2] : 0.5 * ((double)ts[reps / 2 - 1] + ts[reps / 2]);
}

static void push_unique(std::vector<int64_t> &v, int64_t x, int64_t lo, int64_t hi)
{
    x = x < lo ? lo : (x > hi ? hi : x);
    for (int64_t y : v)
        if (y == x)
            return;
    v.push_back(x);
}

std::string window_tune_key(int mode, const Window &win, int64_t rows, int64_t W)
{
    return tune_key(device_tag().c_str(), "window", mode, win.h, win.w, rows, W);
}

bool tune_window(int mode, const Image &g, const Window &win, int64_t row0, int64_t row1, bool pipe,
                 const std::function<cudaError_t()> &launch, cudaStream_t stream, TuneCfg &best)
{
    const int64_t rows = row1 - row0;
    const int64_t th0 = one_wave_tile_rows(rows, g.W);
    std::vector<int64_t> ths;
    push_unique(ths, th0, 1, rows);
    push_unique(ths, th0 + 1, 1, rows);
    push_unique(ths, th0 + 2, 1, rows);
    push_unique(ths, (th0 * 5 + 3) / 4, 1, rows);
    push_unique(ths, (th0 * 3 + 1) / 2, 1, rows);
    push_unique(ths, 2 * th0, 1, rows);
    const float edges[4] = {(float)default_edge_fraction(pipe), pipe ? 0.6f : 0.65f, 0.82f, 1.0f};
    const int nstripe = stripes_allowed(win.h) ? 2 : 1;
    double best_ms = -1.0;
    for (int st = 0; st < nstripe; st++) {
        for (int64_t th : ths) {
            for (int e = 0; e < (st ? 1 : 4); e++) {  // stripe launches use uniform tiles
                TuneCfg c;
                c.tile_h = (int32_t)th;
                c.edge = st ? 1.0f : edges[e];
                c.stripes = st;
                TuneScope scope(&c);
                const double ms = time_on(stream, 9, launch);
                if (ms > 0.0 && (best_ms < 0.0 || ms < best_ms)) {
                    best_ms = ms;
                    best = c;
                    best.us = (float)(ms * 1e3);
                }
            }
        }
    }
    return best_ms > 0.0;
}

bool tune_quantile(const Image &g, const Window &win, const std::function<cudaError_t()> &launch,
                   cudaStream_t stream, TuneCfg &best)
{
    const int64_t th0 = quantile_band_rows(g.H, g.W, win.h);
    std::vector<int64_t> ths;
    push_unique(ths, th0, 1, g.H);
    push_unique(ths, (th0 * 3 + 3) / 4, 1, g.H);
    push_unique(ths, (th0 * 5 + 3) / 4, 1, g.H);
    push_unique(ths, (th0 * 3 + 1) / 2, 1, g.H);
    push_unique(ths, 2 * th0, 1, g.H);
    double best_ms = -1.0;
    for (int64_t th : ths) {
        TuneCfg c;
        c.tile_h = (int32_t)th;
        c.edge = 1.0f;
        c.stripes = -1;
        TuneScope scope(&c);
        const double ms = time_on(stream, 9, launch);
        if (ms > 0.0 && (best_ms < 0.0 || ms < best_ms)) {
            best_ms = ms;
            best = c;
            best.us = (float)(ms * 1e3);
        }
    }
    return best_ms > 0.0;
}

int quantile_class(int32_t q_num, int32_t q_den)
{
    // the walk of Q depends on where the rank falls: low, middle or high
    const double q = (double)q_num / (double)q_den;
    return q < 0.25 ? 0 : (q <= 0.75 ? 1 : 2);
}

std::string quantile_tune_key(int32_t q_num, int32_t q_den, const Window &win, int64_t H, int64_t W)
{
    return tune_key(device_tag().c_str(), "quantile", quantile_class(q_num, q_den), win.h, win.w, H, W);
}

std::string batch_tune_key(int mode)
{
    return tune_key(device_tag().c_str(), "batch", mode, 0, 0, 0, 0);
}

}  // namespace bz

// ------------------------------------------------------------ C ABI --
extern "C" {

int32_t bz_tune_key(const char *gpu, const char *kernel, int32_t cls, int32_t h, int32_t w, int64_t H,
                    int64_t W, char *buf, int32_t len)
{
    if (!gpu || !kernel || !buf || len < 1)
        return -1;
    const std::string k = bz::tune_key(gpu, kernel, cls, h, w, H, W);
    if ((int64_t)k.size() + 1 > len)
        return -1;
    memcpy(buf, k.c_str(), k.size() + 1);
    return (int32_t)k.size();
}

int32_t bz_tune_get(const char *key, int32_t *tile_h, float *edge, int32_t *stripes, float *us)
{
    if (!key)
        return -1;
    bz::TuneCfg c;
    if (!bz::tune_get(key, c))
        return 0;
    if (tile_h)
        *tile_h = c.tile_h;
    if (edge)
        *edge = c.edge;
    if (stripes)
        *stripes = c.stripes;
    if (us)
        *us = c.us;
    return 1;
}

int32_t bz_tune_set(const char *key, int32_t tile_h, float edge, int32_t stripes, float us)
{
    if (!key || tile_h < 0 || !(edge >= 0.0f && edge <= 1.0f) || stripes < -1 || stripes > 64)
        return -1;
    bz::TuneCfg c;
    c.tile_h = tile_h;
    c.edge = edge;
    c.stripes = stripes;
    c.us = us;
    bz::tune_put(key, c, false);
    return 0;
}

int32_t bz_tune_load(const char *path)
{
    std::lock_guard<std::mutex> lk(bz::g_tune_mu);
    bz::g_tune_loaded = true;
    bz::g_tune_path = (path && *path) ? path : bz::default_cache_path();
    bz::g_tune.clear();
    std::string text;
    std::map<std::string, bz::TuneCfg> m;
    if (!bz::read_file(bz::g_tune_path, text))
        return -1;
    if (!bz::parse_cache(text, m))
        return -2;
    bz::g_tune.swap(m);
    return (int32_t)bz::g_tune.size();
}

int32_t bz_tune_save(const char *path)
{
    std::lock_guard<std::mutex> lk(bz::g_tune_mu);
    bz::load_locked();
    return bz::save_locked((path && *path) ? std::string(path) : bz::g_tune_path) ? 0 : -1;
}

void bz_tune_clear(void)
{
    std::lock_guard<std::mutex> lk(bz::g_tune_mu);
    bz::g_tune_loaded = true;
    bz::g_tune.clear();
}

int32_t bz_tune_window_plan(const char *gpu, int32_t precision, int64_t H, int64_t W, int32_t h, int32_t w,
                            int32_t sms, int64_t *out)
{
    if (!gpu || !out || H < 1 || W < 1 || h < 1 || w < 1 || h > 511 || w > 511 || sms < 1)
        return -1;
    if (precision < 0 || precision > 2)
        return -1;
    const int mode = precision == 0 ? bz::MODE_FP64 : (precision == 1 ? bz::MODE_FP32 : bz::MODE_FP64_DIRECT);
    const bz::Window win = bz::make_window(h, w);
    bz::TuneCfg c;
    const bool cached = bz::tune_env() != 0 && bz::tune_get(bz::tune_key(gpu, "window", mode, h, w, H, W), c);
    bz::TuneScope scope(cached ? &c : nullptr);
    return bz::plan_window_launch(H, W, win, sms, true, out) == 0 ? (cached ? 1 : 0) : -1;
}

}  // extern "C"
