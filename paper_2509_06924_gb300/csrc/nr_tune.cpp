// nr_tune.cpp -- the persisted autotune cache: a small JSON file mapping a
// key (GPU, SM count, mode, quadrature order, register bucket, size class,
// tuner version) to the launch shape the autotuner chose.  Host code only.
//
// File layout (written by nr_tune_cache_put, read back by _get):
//   {"version": 1, "entries": {"<key>": {"paired": 1, "tile_q": 12,
//    "ctas_per_sm": 4, "ms": 1.25}, ...}}
// The reader is a small recursive-descent parser of exactly this shape of
// JSON (objects, strings without escapes, numbers); anything else makes the
// file unreadable, which the library treats as an empty cache.
#include <algorithm>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "nr.h"

namespace nrimpl {
void record_error(const char *msg); // nr_api.cpp: message for nr_last_error()
}

namespace {

using Entries = std::map<std::string, nr_tune_entry>;
std::mutex g_tune_mutex;

struct Parser {
    const char *p, *end;
    void ws()
    {
        while (p < end && std::isspace((unsigned char)*p)) ++p;
    }
    bool eat(char c)
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
        const char *q = ++p;
        while (p < end && *p != '"') {
            if (*p == '\\') return false; // escapes are never written
            ++p;
        }
        if (p >= end) return false;
        out.assign(q, p - q);
        ++p;
        return true;
    }
    bool num(double &v)
    {
        ws();
        char *stop = nullptr;
        const std::string tmp(p, std::min<size_t>(end - p, 64));
        v = std::strtod(tmp.c_str(), &stop);
        if (stop == tmp.c_str()) return false;
        p += stop - tmp.c_str();
        return true;
    }
    // {"paired": i, "tile_q": i, "ctas_per_sm": i, "ms": x} in any order
    bool entry(nr_tune_entry &e)
    {
        e = nr_tune_entry{};
        if (!eat('{')) return false;
        if (eat('}')) return true;
        do {
            std::string k;
            double v = 0.0;
            if (!str(k) || !eat(':') || !num(v)) return false;
            if (k == "paired") e.paired = (int32_t)v;
            else if (k == "tile_q") e.tile_q = (int32_t)v;
            else if (k == "ctas_per_sm") e.ctas_per_sm = (int32_t)v;
            else if (k == "ms") e.ms = v;
        } while (eat(','));
        return eat('}');
    }
    bool file(Entries &out)
    {
        if (!eat('{')) return false;
        bool have_entries = false;
        if (eat('}')) return false;
        do {
            std::string k;
            if (!str(k) || !eat(':')) return false;
            if (k == "entries") {
                if (!eat('{')) return false;
                if (!eat('}')) {
                    do {
                        std::string key;
                        nr_tune_entry e;
                        if (!str(key) || !eat(':') || !entry(e)) return false;
                        out[key] = e;
                    } while (eat(','));
                    if (!eat('}')) return false;
                }
                have_entries = true;
            } else {
                double v;
                if (!num(v)) return false; // "version": 1
            }
        } while (eat(','));
        return eat('}') && have_entries;
    }
};

bool load(const char *path, Entries &out)
{
    FILE *f = std::fopen(path, "rb");
    if (!f) return false;
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
    std::fclose(f);
    Parser ps{text.data(), text.data() + text.size()};
    Entries tmp;
    if (!ps.file(tmp)) return false;
    out.swap(tmp);
    return true;
}

bool save(const char *path, const Entries &entries)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return false;
    std::fprintf(f, "{\"version\": 1, \"entries\": {");
    bool first = true;
    for (const auto &kv : entries) {
        const nr_tune_entry &e = kv.second;
        std::fprintf(f, "%s\n  \"%s\": {\"paired\": %d, \"tile_q\": %d, \"ctas_per_sm\": %d, \"ms\": %.6g}",
                     first ? "" : ",", kv.first.c_str(), e.paired, e.tile_q, e.ctas_per_sm, e.ms);
        first = false;
    }
    std::fprintf(f, "\n}}\n");
    const bool ok = std::fclose(f) == 0;
    return ok && std::rename(tmp.c_str(), path) == 0;
}

nr_status fail(const char *msg)
{
    nrimpl::record_error(msg);
    return NR_EINVAL;
}

} // namespace

extern "C" {

nr_status nr_tune_cache_get(const char *path, const char *key, nr_tune_entry *entry)
{
    if (!path || !key || !entry) return fail("nr_tune_cache_get: NULL argument");
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    Entries es;
    if (!load(path, es)) return fail("nr_tune_cache_get: cache file absent or unreadable");
    const auto it = es.find(key);
    if (it == es.end()) return fail("nr_tune_cache_get: key not in the cache");
    *entry = it->second;
    return NR_OK;
}

nr_status nr_tune_cache_put(const char *path, const char *key, const nr_tune_entry *entry)
{
    if (!path || !key || !entry) return fail("nr_tune_cache_put: NULL argument");
    if (std::strchr(key, '"') || std::strchr(key, '\\')) return fail("nr_tune_cache_put: key holds '\"' or '\\'");
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    Entries es;
    load(path, es); // a missing or unreadable file starts a new cache
    es[key] = *entry;
    if (!save(path, es)) return fail("nr_tune_cache_put: cannot write the cache file");
    return NR_OK;
}

} // extern "C"
