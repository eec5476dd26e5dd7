// Autotuner of the persistent method and its on-disk cache (host code).
//
// The persistent kernel's tuning (block size, refill threshold, queue chunk,
// and the collision batch size) changes only the order in which lanes do
// their work, never an event's result, so it can be chosen by timing alone. The search is
// a coordinate descent from the context's current tuning: each parameter in turn takes each
// candidate value with the others fixed, and keeps the fastest; two passes.
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "api_internal.h"

using namespace pnuc;

namespace {

int32_t *field(pnuc_tuning &t, int k)
{
    switch (k) {
    case 0: return &t.block_size;
    case 1: return &t.kin_batch;
    case 2: return &t.refill_threshold;
    default: return &t.chunk;
    }
}

std::vector<int32_t> candidates(int k)
{
    switch (k) {
    case 0: return {64, 128, 256};
    case 1: return {1, 8, 16, 24, 32};
    case 2: return {1, 2, 4, 8, 16};
    default: return {64, 256, 1024};
    }
}

// Mean time of `reps` launches after one warm-up, or a negative value on error.
double time_tuning(pnuc_ctx *ctx, pnuc_precision prec, const pnuc_batch *b, const pnuc_output *o, const pnuc_tuning &t,
                   int reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1)
{
    if (launch_batch(ctx, prec, PNUC_PERSISTENT, b, o, s, t, nullptr) != PNUC_OK) return -1.0;
    if (cudaEventRecord(e0, s) != cudaSuccess) return -1.0;
    for (int r = 0; r < reps; ++r)
        if (launch_batch(ctx, prec, PNUC_PERSISTENT, b, o, s, t, nullptr) != PNUC_OK) return -1.0;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
}

// ---- minimal JSON for the cache file: {"<device>": {"fp32": {"key": int, ...}, "fp64": {...}}, ...}
struct Json {
    const char *p;
    void ws()
    {
        while (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t') ++p;
    }
    bool str(std::string &out)
    {
        ws();
        if (*p != '"') return false;
        ++p;
        out.clear();
        while (*p && *p != '"') {
            if (*p == '\\' && p[1]) ++p;
            out += *p++;
        }
        if (*p != '"') return false;
        ++p;
        return true;
    }
    bool integer(long long &v)
    {
        ws();
        char *end = nullptr;
        v = strtoll(p, &end, 10);
        if (end == p) return false;
        p = end;
        return true;
    }
    bool lit(char c)
    {
        ws();
        if (*p != c) return false;
        ++p;
        return true;
    }
};

const char *kKeys[5] = {"block_size", "blocks_per_sm", "refill_threshold", "chunk", "kin_batch"};

int32_t *by_name(pnuc_tuning &t, const std::string &k)
{
    if (k == kKeys[0]) return &t.block_size;
    if (k == kKeys[1]) return &t.blocks_per_sm;
    if (k == kKeys[2]) return &t.refill_threshold;
    if (k == kKeys[3]) return &t.chunk;
    if (k == kKeys[4]) return &t.kin_batch;
    return nullptr;
}

struct Entry {
    std::string device;
    bool has[2] = {false, false};
    pnuc_tuning t[2];
};

// Parses the cache; returns false on malformed input.
bool parse_cache(const std::string &text, std::vector<Entry> &out)
{
    Json j{text.c_str()};
    if (!j.lit('{')) return false;
    if (j.lit('}')) return true;
    do {
        Entry e;
        if (!j.str(e.device) || !j.lit(':') || !j.lit('{')) return false;
        if (!j.lit('}')) {
            do {
                std::string prec;
                if (!j.str(prec) || !j.lit(':') || !j.lit('{')) return false;
                int pi = prec == "fp64" ? 1 : (prec == "fp32" ? 0 : -1);
                pnuc_tuning t{};
                if (!j.lit('}')) {
                    do {
                        std::string k;
                        long long v;
                        if (!j.str(k) || !j.lit(':') || !j.integer(v)) return false;
                        if (int32_t *f = by_name(t, k)) *f = (int32_t)v;
                    } while (j.lit(','));
                    if (!j.lit('}')) return false;
                }
                if (pi >= 0) {
                    e.t[pi] = t;
                    e.has[pi] = true;
                }
            } while (j.lit(','));
            if (!j.lit('}')) return false;
        }
        out.push_back(e);
    } while (j.lit(','));
    return j.lit('}');
}

std::string escape(const std::string &s)
{
    std::string o;
    for (char c : s) {
        if (c == '"' || c == '\\') o += '\\';
        o += c;
    }
    return o;
}

}  // namespace

extern "C" {

pnuc_status pnuc_autotune(pnuc_ctx *ctx, pnuc_precision precision, const pnuc_batch *batch, const pnuc_output *out,
                          int32_t reps, pnuc_tuning *best, double *best_ms, void *stream)
{
    pnuc_status st = check_batch(ctx, precision, PNUC_PERSISTENT, batch, out);
    if (st != PNUC_OK) return st;
    if (batch->n == 0) return fail(ctx, PNUC_ERR_ARG, "autotune needs a non-empty batch");
    if (reps < 1 || reps > 100) return fail(ctx, PNUC_ERR_ARG, "reps %d not in [1, 100]", reps);
    cudaStream_t s = (cudaStream_t)stream;
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    cudaEvent_t e0, e1;
    CU(ctx, cudaEventCreate(&e0));
    CU(ctx, cudaEventCreate(&e1));
    pnuc_tuning cur = ctx->tuning[tuning_slot(precision)];
    cur.blocks_per_sm = 32;  // the launch clamps to the kernel's occupancy
    double cur_ms = time_tuning(ctx, precision, batch, out, cur, reps, s, e0, e1);
    for (int pass = 0; pass < 2 && cur_ms > 0; ++pass) {
        for (int k = 0; k < 4; ++k) {
            for (int32_t v : candidates(k)) {
                pnuc_tuning t = cur;
                *field(t, k) = v;
                if (*field(cur, k) == v || check_tuning(nullptr, &t) != PNUC_OK) continue;
                double ms = time_tuning(ctx, precision, batch, out, t, reps, s, e0, e1);
                if (ms > 0 && ms < cur_ms) {
                    cur_ms = ms;
                    cur = t;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!(cur_ms > 0)) return fail(ctx, PNUC_ERR_CUDA, "autotune launch failed: %s", ctx->err);
    ctx->tuning[tuning_slot(precision)] = cur;
    if (best) *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return PNUC_OK;
}

pnuc_status pnuc_save_tuning(pnuc_ctx *ctx, const char *path)
{
    if (!ctx || !path) return fail(ctx, PNUC_ERR_ARG, "null argument");
    std::vector<Entry> entries;
    if (FILE *f = fopen(path, "rb")) {
        std::string text;
        char buf[4096];
        size_t k;
        while ((k = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
        fclose(f);
        if (!parse_cache(text, entries)) entries.clear();  // a malformed cache is replaced
    }
    Entry *mine = nullptr;
    for (auto &e : entries)
        if (e.device == ctx->device_name) mine = &e;
    if (!mine) {
        entries.push_back(Entry{});
        mine = &entries.back();
        mine->device = ctx->device_name;
    }
    for (int p = 0; p < 2; ++p) {
        mine->t[p] = ctx->tuning[p];
        mine->has[p] = true;
    }
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(ctx, PNUC_ERR_ARG, "cannot write %s", tmp.c_str());
    fprintf(f, "{\n");
    for (size_t i = 0; i < entries.size(); ++i) {
        fprintf(f, "  \"%s\": {", escape(entries[i].device).c_str());
        bool first = true;
        for (int p = 0; p < 2; ++p) {
            if (!entries[i].has[p]) continue;
            pnuc_tuning &t = entries[i].t[p];
            fprintf(f, "%s\n    \"%s\": {", first ? "" : ",", p ? "fp64" : "fp32");
            for (int k = 0; k < 5; ++k) fprintf(f, "%s\"%s\": %d", k ? ", " : "", kKeys[k], *by_name(t, kKeys[k]));
            fprintf(f, "}");
            first = false;
        }
        fprintf(f, "\n  }%s\n", i + 1 < entries.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    if (rename(tmp.c_str(), path) != 0) return fail(ctx, PNUC_ERR_ARG, "cannot replace %s", path);
    return PNUC_OK;
}

pnuc_status pnuc_load_tuning(pnuc_ctx *ctx, const char *path)
{
    if (!ctx || !path) return fail(ctx, PNUC_ERR_ARG, "null argument");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(ctx, PNUC_ERR_RANGE, "no tuning cache at %s", path);
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
    fclose(f);
    std::vector<Entry> entries;
    if (!parse_cache(text, entries)) return fail(ctx, PNUC_ERR_ARG, "malformed tuning cache %s", path);
    for (auto &e : entries) {
        if (e.device != ctx->device_name) continue;
        for (int p = 0; p < 2; ++p) {
            if (!e.has[p]) continue;
            pnuc_status st = check_tuning(ctx, &e.t[p]);
            if (st != PNUC_OK) return st;
        }
        for (int p = 0; p < 2; ++p)
            if (e.has[p]) ctx->tuning[p] = e.t[p];
        return PNUC_OK;
    }
    return fail(ctx, PNUC_ERR_RANGE, "tuning cache %s has no entry for %s", path, ctx->device_name);
}

}  // extern "C"
