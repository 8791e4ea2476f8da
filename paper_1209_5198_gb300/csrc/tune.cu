// Autotuner of the decomposition and its cache (gf2_tune_* and
// gf2_decompose_autotune of include/gf2.h).
//
// The paper tunes its block and table sizes by hand for one CPU (Sections
// 6.1 and 7); here the choices that change only speed -- the width of the
// trailing updates (one 64-column block or a pair, Section 5's wide panel),
// the bits of their Four Russians tables (Section 6) and the schedule of the
// launches -- are timed on the device itself and remembered per (device,
// shape bucket).  A decomposition called with automatic options takes the
// entry of its bucket when there is one.  The entries can be saved to and
// loaded from a JSON file, so a tuned process can hand them to the next one.
//
// Shape bucket: the powers of two at or above the row and column counts
// (at least 64 each), so 20000 x 30000 shares the 32768 x 32768 entry.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include <cstdio>
#include <cstring>

#include "../../include/gf2.h"
#include "gf2_internal.cuh"

namespace gf2 {
namespace {

std::mutex g_tune_mu;
std::vector<gf2_tune_entry> g_tune;  // guarded by g_tune_mu

int64_t bucket_of(int64_t x)
{
    int64_t b = 64;
    while (b < x && b < ((int64_t)1 << 40)) b <<= 1;
    return b;
}

bool same_slot(const gf2_tune_entry &a, const gf2_tune_entry &b)
{
    return a.kind == b.kind && a.bucket_n == b.bucket_n && a.bucket_m == b.bucket_m &&
           strncmp(a.device, b.device, sizeof(a.device)) == 0;
}

bool entry_ok(const gf2_tune_entry &e)
{
    if (memchr(e.device, 0, sizeof(e.device)) == nullptr || e.device[0] == 0) return false;
    for (const char *c = e.device; *c; ++c)  // the JSON file writes the key without escapes
        if (*c == '"' || *c == '\\' || (unsigned char)*c < 0x20) return false;
    if (e.kind != GF2_TUNE_DECOMPOSE || e.reserved != 0) return false;
    if (e.bucket_n < 64 || e.bucket_m < 64 || bucket_of(e.bucket_n) != e.bucket_n || bucket_of(e.bucket_m) != e.bucket_m)
        return false;
    if (!(e.ms >= 0.0)) return false;
    return gf2_opts_check(&e.opts) == GF2_OK;
}

// ------------------------------------------------------------ JSON
// The file is one object: {"gf2_tune": 1, "entries": [ {...}, ... ]}; an
// entry has the string "device", the string "kind" ("decompose") and the
// numbers bucket_n, bucket_m, panel_w, table_c, tile_words, backend,
// schedule, strassen_cutoff, batched_c8_from and ms.  The reader accepts
// that shape with any whitespace and key order; anything else is an error.
struct Json {
    const char *p, *end;
    void ws()
    {
        while (p < end && (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r')) ++p;
    }
    bool lit(char c)
    {
        ws();
        if (p < end && *p == c) {
            ++p;
            return true;
        }
        return false;
    }
    bool str(std::string &out)
    {
        ws();
        if (p >= end || *p != '"') return false;
        ++p;
        out.clear();
        while (p < end && *p != '"') {
            if (*p == '\\') {
                if (++p >= end) return false;
                if (*p != '"' && *p != '\\' && *p != '/') return false;
            }
            out.push_back(*p++);
        }
        if (p >= end) return false;
        ++p;
        return true;
    }
    bool num(double &out)
    {
        ws();
        char *e = nullptr;
        std::string tmp(p, (size_t)std::min<ptrdiff_t>(end - p, 64));
        out = strtod(tmp.c_str(), &e);
        if (e == tmp.c_str()) return false;
        p += e - tmp.c_str();
        return true;
    }
};

bool parse_entry(Json &js, gf2_tune_entry &e)
{
    memset(&e, 0, sizeof(e));
    if (!js.lit('{')) return false;
    bool have_dev = false, have_kind = false, first = true;
    int seen = 0;
    for (;;) {
        if (js.lit('}')) break;
        if (!first && !js.lit(',')) return false;
        first = false;
        std::string key;
        if (!js.str(key) || !js.lit(':')) return false;
        if (key == "device" || key == "kind") {
            std::string v;
            if (!js.str(v)) return false;
            if (key == "device") {
                if (v.empty() || v.size() >= sizeof(e.device)) return false;
                memcpy(e.device, v.c_str(), v.size() + 1);
                have_dev = true;
            } else {
                if (v != "decompose") return false;
                e.kind = GF2_TUNE_DECOMPOSE;
                have_kind = true;
            }
            continue;
        }
        double v = 0;
        if (!js.num(v)) return false;
        const int64_t iv = (int64_t)v;
        if (key == "ms") e.ms = v;
        else if ((double)iv != v) return false;
        else if (key == "bucket_n") e.bucket_n = iv;
        else if (key == "bucket_m") e.bucket_m = iv;
        else if (key == "panel_w") e.opts.panel_w = (int32_t)iv;
        else if (key == "table_c") e.opts.table_c = (int32_t)iv;
        else if (key == "tile_words") e.opts.tile_words = (int32_t)iv;
        else if (key == "backend") e.opts.backend = (int32_t)iv;
        else if (key == "schedule") e.opts.schedule = (int32_t)iv;
        else if (key == "strassen_cutoff") e.opts.strassen_cutoff = iv;
        else if (key == "batched_c8_from") e.opts.batched_c8_from = iv;
        else return false;
        ++seen;
    }
    return have_dev && have_kind && seen >= 3 && entry_ok(e);
}

bool parse_file(const std::string &text, std::vector<gf2_tune_entry> &out)
{
    Json js{text.data(), text.data() + text.size()};
    if (!js.lit('{')) return false;
    bool have_entries = false, first = true;
    for (;;) {
        if (js.lit('}')) break;
        if (!first && !js.lit(',')) return false;
        first = false;
        std::string key;
        if (!js.str(key) || !js.lit(':')) return false;
        if (key == "gf2_tune") {
            double v = 0;
            if (!js.num(v) || v != 1.0) return false;
        } else if (key == "entries") {
            if (!js.lit('[')) return false;
            bool f2 = true;
            for (;;) {
                if (js.lit(']')) break;
                if (!f2 && !js.lit(',')) return false;
                f2 = false;
                gf2_tune_entry e;
                if (!parse_entry(js, e)) return false;
                out.push_back(e);
            }
            have_entries = true;
        } else {
            return false;
        }
    }
    js.ws();
    return have_entries && js.p == js.end;
}

void put_locked(const gf2_tune_entry &e)
{
    for (auto &x : g_tune)
        if (same_slot(x, e)) {
            x = e;
            return;
        }
    g_tune.push_back(e);
}

// ------------------------------------------------------------ tuning input
// splitmix64 (Steele, Lea, Flood 2014) of a counter: a uniform random word
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// words (i, q) of an n x m matrix in column blocks (ld = n), padding zero
__global__ void k_tune_fill(uint64_t *A, int64_t n, int64_t mu, uint64_t last_mask)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * mu) return;
    const int64_t q = e / n;
    const uint64_t w = mix64(0x1209519800000000ull ^ (uint64_t)e);
    A[e] = q == mu - 1 ? (w & last_mask) : w;
}

}  // namespace

bool tuned_decompose_opts(int64_t n, int64_t m, gf2_opts *out)
{
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (g_tune.empty()) return false;  // nothing tuned: no device query at all
    }
    gf2_tune_entry key{};
    if (gf2_tune_device_key(key.device, sizeof(key.device)) != GF2_OK) return false;
    key.kind = GF2_TUNE_DECOMPOSE;
    key.bucket_n = bucket_of(n);
    key.bucket_m = bucket_of(m);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto &x : g_tune)
        if (same_slot(x, key)) {
            *out = x.opts;
            return true;
        }
    return false;
}

}  // namespace gf2

using namespace gf2;

extern "C" {

int gf2_tune_device_key(char *out, int64_t len)
{
    if (!out || len < 1) return GF2_ERR_ARG;
    // the key of each device is made once (reading the device properties is
    // slow) and then copied: every decomposition with automatic options asks
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static char keys[kMaxDev][sizeof(((gf2_tune_entry *)nullptr)->device)] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return GF2_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(mu);
    char *buf = keys[dev];
    if (!buf[0]) {
        int sms = 0;
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return GF2_ERR_CUDA;
        }
        snprintf(buf, sizeof(keys[0]), "%s sm%d cc%d.%d", prop.name, sms, prop.major, prop.minor);
        for (char *c = buf; *c; ++c)
            if (*c == '"' || *c == '\\' || (unsigned char)*c < 0x20) *c = '_';  // nothing the JSON file would escape
    }
    if ((int64_t)strlen(buf) >= len) return GF2_ERR_ARG;
    memcpy(out, buf, strlen(buf) + 1);
    return GF2_OK;
}

int gf2_tune_put(const gf2_tune_entry *e)
{
    if (!e || !entry_ok(*e)) return GF2_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    put_locked(*e);
    return GF2_OK;
}

int gf2_tune_lookup(const char *device, int32_t kind, int64_t n, int64_t m, gf2_tune_entry *out, int *found)
{
    if (!device || !out || !found || n < 0 || m < 0 || kind != GF2_TUNE_DECOMPOSE) return GF2_ERR_ARG;
    gf2_tune_entry key{};
    const size_t dl = strnlen(device, sizeof(key.device));
    if (dl == 0 || dl >= sizeof(key.device)) return GF2_ERR_ARG;
    memcpy(key.device, device, dl);
    key.kind = kind;
    key.bucket_n = bucket_of(n);
    key.bucket_m = bucket_of(m);
    *found = 0;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto &x : g_tune)
        if (same_slot(x, key)) {
            *out = x;
            *found = 1;
            break;
        }
    return GF2_OK;
}

int64_t gf2_tune_count(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    return (int64_t)g_tune.size();
}

int gf2_tune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
    return GF2_OK;
}

int gf2_tune_save(const char *path)
{
    if (!path) return GF2_ERR_ARG;
    std::vector<gf2_tune_entry> snap;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        snap = g_tune;
    }
    FILE *f = fopen(path, "w");
    if (!f) return GF2_ERR_ARG;
    fprintf(f, "{\"gf2_tune\": 1, \"entries\": [");
    for (size_t i = 0; i < snap.size(); ++i) {
        const gf2_tune_entry &e = snap[i];
        fprintf(f,
                "%s\n  {\"device\": \"%s\", \"kind\": \"decompose\", \"bucket_n\": %lld, \"bucket_m\": %lld, "
                "\"panel_w\": %d, \"table_c\": %d, \"tile_words\": %d, \"backend\": %d, \"schedule\": %d, "
                "\"strassen_cutoff\": %lld, \"batched_c8_from\": %lld, \"ms\": %.6f}",
                i ? "," : "", e.device, (long long)e.bucket_n, (long long)e.bucket_m, e.opts.panel_w, e.opts.table_c,
                e.opts.tile_words, e.opts.backend, e.opts.schedule, (long long)e.opts.strassen_cutoff,
                (long long)e.opts.batched_c8_from, e.ms);
    }
    fprintf(f, "\n]}\n");
    return fclose(f) == 0 ? GF2_OK : GF2_ERR_ARG;
}

int gf2_tune_load(const char *path)
{
    if (!path) return GF2_ERR_ARG;
    FILE *f = fopen(path, "r");
    if (!f) return GF2_ERR_ARG;
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof(buf), f)) > 0 && text.size() < (1u << 24)) text.append(buf, k);
    fclose(f);
    std::vector<gf2_tune_entry> entries;
    if (!parse_file(text, entries)) return GF2_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto &e : entries) put_locked(e);
    return GF2_OK;
}

int gf2_decompose_autotune(int64_t n, int64_t m, int want_factors, gf2_tune_entry *best, void *stream)
{
    if (!best || n < 1 || m < 1 || n >= (1ll << 31) || m >= (1ll << 31)) return GF2_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gf2_tune_entry e{};
    int st = gf2_tune_device_key(e.device, sizeof(e.device));
    if (st) return st;
    e.kind = GF2_TUNE_DECOMPOSE;
    e.bucket_n = bucket_of(n);
    e.bucket_m = bucket_of(m);
    // the candidates: one block or a pair per update, 4- or 8-bit tables,
    // and for pairs the three schedules
    std::vector<gf2_opts> cand;
    for (int tc : {8, 4}) {
        gf2_opts o{};
        o.panel_w = 64;
        o.table_c = tc;
        cand.push_back(o);
        for (int sch : {GF2_SCHEDULE_STREAMS, GF2_SCHEDULE_PERSISTENT, GF2_SCHEDULE_SPLIT}) {
            gf2_opts p{};
            p.panel_w = 128;
            p.table_c = tc;
            p.schedule = sch;
            cand.push_back(p);
        }
    }
    const int64_t mu = (m + 63) / 64, k = n < m ? n : m, kw = (k + 63) / 64;
    const size_t ws_bytes = gf2_decompose_workspace_bytes(n, m, want_factors ? 1 : 0);
    uint64_t *A = nullptr, *L = nullptr, *E = nullptr;
    int32_t *perm = nullptr, *piv = nullptr;
    int64_t *rank = nullptr;
    void *ws = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto release = [&]() {
        cudaStreamSynchronize(s);
        cudaFree(A);
        cudaFree(L);
        cudaFree(E);
        cudaFree(perm);
        cudaFree(piv);
        cudaFree(rank);
        cudaFree(ws);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&A, (size_t)n * mu * 8) != cudaSuccess || cudaMalloc(&perm, (size_t)n * 4) != cudaSuccess ||
        cudaMalloc(&piv, (size_t)k * 4) != cudaSuccess || cudaMalloc(&rank, 8) != cudaSuccess ||
        cudaMalloc(&ws, ws_bytes) != cudaSuccess ||
        (want_factors && (cudaMalloc(&L, (size_t)n * kw * 8) != cudaSuccess ||
                          cudaMalloc(&E, (size_t)k * mu * 8) != cudaSuccess))) {
        cudaGetLastError();
        release();
        return GF2_ERR_NOMEM;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        release();
        return GF2_ERR_CUDA;
    }
    const uint64_t last_mask = (m % 64) ? ((1ull << (m % 64)) - 1) : ~0ull;
    k_tune_fill<<<(unsigned)((n * mu + 255) / 256), 256, 0, s>>>(A, n, mu, last_mask);
    if (cudaGetLastError() != cudaSuccess) {
        release();
        return GF2_ERR_CUDA;
    }
    gf2_mat Am{A, n, m, n}, Lm{L, n, k, n}, Em{E, k, m, k};
    double best_ms = 1e30;
    for (const gf2_opts &o : cand) {
        // three untimed calls (the second captures the graph the later ones replay), then the best of three
        float t = 1e30f;
        for (int it = 0; it < 6 && !st; ++it) {
            if (it >= 3 && cudaEventRecord(e0, s) != cudaSuccess) st = GF2_ERR_CUDA;
            if (!st)
                st = gf2_decompose_ex(&Am, perm, piv, rank, want_factors ? &Lm : nullptr, want_factors ? &Em : nullptr,
                                      GF2_NOCHECK, &o, ws, ws_bytes, s);
            if (!st && it >= 3) {
                float ms = 0.f;
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                    st = GF2_ERR_CUDA;
                else if (ms < t)
                    t = ms;
            }
        }
        int64_t r = 0;
        if (!st && cudaMemcpyAsync(&r, rank, 8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess && r < 0)
            st = GF2_ERR_TIMEOUT;
        if (st) break;
        if (t < best_ms) {
            best_ms = t;
            e.opts = o;
        }
    }
    release();
    if (st) return st;
    e.ms = best_ms;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        put_locked(e);
    }
    *best = e;
    return GF2_OK;
}

}  // extern "C"
