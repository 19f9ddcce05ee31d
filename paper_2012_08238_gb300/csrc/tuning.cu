// Measured plan sizes per size class (the autotuner's cache), read from JSON.
//
// The paper tunes its parameters "to balance time efficiency and
// robustness" and gives no values; this library's tuner
// (paper_2012_08238_gb300/tune.py) measures, per size class, the fastest
// (B, w, L) whose L1 error and support recall match the fixed rule's, and
// writes them as
//   {"version": 1, ..., "classes": [{"logN": n, "K_lo": a, "K_hi": b,
//     "snr_lo": s0, "snr_hi": s1, "B_per_K": r, "w_extra": e, "L": l, ...}]}
// (snr_lo / snr_hi null: noiseless signals).  A class covers N = 2^n,
// a <= K <= b and s0 <= SNR < s1; it sets B = the smallest power of two
// >= r K (within the size rule's bounds), w = B (log2 N + e), L = l.  Other
// keys are ignored.  sfft_suggest_params consults the loaded classes first.
#include <ctype.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "sfft_internal.cuh"

namespace sfft {

namespace {

struct TuneClass {
    int logN;
    int64_t K_lo, K_hi;
    bool noiseless;
    double snr_lo, snr_hi;
    int64_t B_per_K, w_extra;
    int32_t L;
};

std::mutex g_tune_mu;
std::vector<TuneClass> g_classes;

// A small JSON reader: objects, arrays, numbers, strings, true/false/null.
struct Json {
    enum Kind { kNull, kBool, kNum, kStr, kArr, kObj } kind = kNull;
    double num = 0.0;
    bool b = false;
    std::string str;
    std::vector<Json> items;                              // array
    std::vector<std::pair<std::string, Json>> members;    // object
    const Json *get(const char *k) const {
        for (const auto &m : members)
            if (m.first == k) return &m.second;
        return nullptr;
    }
};

struct Parser {
    const char *p, *end;
    std::string err;
    void ws() {
        while (p < end && isspace((unsigned char)*p)) ++p;
    }
    bool fail(const char *m) {
        if (err.empty()) err = m;
        return false;
    }
    bool lit(const char *w) {
        const size_t n = strlen(w);
        if ((size_t)(end - p) < n || strncmp(p, w, n) != 0) return false;
        p += n;
        return true;
    }
    bool string(std::string &out) {
        if (p >= end || *p != '"') return fail("expected a string");
        ++p;
        while (p < end && *p != '"') {
            if (*p == '\\') {
                ++p;
                if (p >= end) return fail("unterminated escape");
                const char c = *p;
                out.push_back(c == 'n' ? '\n' : c == 't' ? '\t' : c);  // (\uXXXX is not used by the cache)
            } else {
                out.push_back(*p);
            }
            ++p;
        }
        if (p >= end) return fail("unterminated string");
        ++p;
        return true;
    }
    bool value(Json &v, int depth) {
        if (depth > 32) return fail("nesting too deep");
        ws();
        if (p >= end) return fail("unexpected end");
        if (*p == '{') {
            ++p;
            v.kind = Json::kObj;
            ws();
            if (p < end && *p == '}') {
                ++p;
                return true;
            }
            for (;;) {
                ws();
                std::string k;
                if (!string(k)) return false;
                ws();
                if (p >= end || *p != ':') return fail("expected ':'");
                ++p;
                Json m;
                if (!value(m, depth + 1)) return false;
                v.members.emplace_back(k, m);
                ws();
                if (p < end && *p == ',') {
                    ++p;
                    continue;
                }
                if (p < end && *p == '}') {
                    ++p;
                    return true;
                }
                return fail("expected ',' or '}'");
            }
        }
        if (*p == '[') {
            ++p;
            v.kind = Json::kArr;
            ws();
            if (p < end && *p == ']') {
                ++p;
                return true;
            }
            for (;;) {
                Json it;
                if (!value(it, depth + 1)) return false;
                v.items.push_back(it);
                ws();
                if (p < end && *p == ',') {
                    ++p;
                    continue;
                }
                if (p < end && *p == ']') {
                    ++p;
                    return true;
                }
                return fail("expected ',' or ']'");
            }
        }
        if (*p == '"') {
            v.kind = Json::kStr;
            return string(v.str);
        }
        if (lit("true")) {
            v.kind = Json::kBool;
            v.b = true;
            return true;
        }
        if (lit("false")) {
            v.kind = Json::kBool;
            return true;
        }
        if (lit("null")) return true;
        char *q = nullptr;
        const std::string tok(p, (size_t)std::min<ptrdiff_t>(end - p, 64));
        v.num = strtod(tok.c_str(), &q);
        if (q == tok.c_str()) return fail("expected a value");
        v.kind = Json::kNum;
        p += q - tok.c_str();
        return true;
    }
};

bool num_of(const Json &o, const char *k, double &out) {
    const Json *v = o.get(k);
    if (!v || v->kind != Json::kNum) return false;
    out = v->num;
    return true;
}

}  // namespace

bool tuning_lookup(int logN, int64_t K, double snr_db, int64_t *B_per_K, int64_t *w_extra, int32_t *L) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const bool noiseless = std::isnan(snr_db);
    for (const TuneClass &c : g_classes) {
        if (c.logN != logN || K < c.K_lo || K > c.K_hi || c.noiseless != noiseless) continue;
        if (!noiseless && (snr_db < c.snr_lo || snr_db >= c.snr_hi)) continue;
        *B_per_K = c.B_per_K;
        *w_extra = c.w_extra;
        *L = c.L;
        return true;
    }
    return false;
}

}  // namespace sfft

using namespace sfft;

extern "C" sfft_status sfft_tuning_load(const char *path) {
    if (!path) {
        set_error("NULL path");
        return SFFT_EINVAL;
    }
    FILE *fh = fopen(path, "rb");
    if (!fh) {
        set_error(std::string("cannot open tuning cache ") + path);
        return SFFT_EINVAL;
    }
    std::string text;
    char buf[65536];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), fh)) > 0) text.append(buf, n);
    fclose(fh);
    Parser ps{text.data(), text.data() + text.size(), {}};
    Json root;
    if (!ps.value(root, 0) || root.kind != Json::kObj) {
        set_error("tuning cache: " + (ps.err.empty() ? std::string("not a JSON object") : ps.err));
        return SFFT_EINVAL;
    }
    double ver = 0;
    const Json *cls = root.get("classes");
    if (!num_of(root, "version", ver) || ver != 1.0 || !cls || cls->kind != Json::kArr) {
        set_error("tuning cache: needs \"version\": 1 and a \"classes\" array");
        return SFFT_EINVAL;
    }
    std::vector<TuneClass> out;
    for (const Json &c : cls->items) {
        double logN, klo, khi, bpk, wex, L;
        if (c.kind != Json::kObj || !num_of(c, "logN", logN) || !num_of(c, "K_lo", klo) || !num_of(c, "K_hi", khi) ||
            !num_of(c, "B_per_K", bpk) || !num_of(c, "w_extra", wex) || !num_of(c, "L", L)) {
            set_error("tuning cache: a class lacks logN, K_lo, K_hi, B_per_K, w_extra or L");
            return SFFT_EINVAL;
        }
        TuneClass t;
        t.logN = (int)logN;
        t.K_lo = (int64_t)klo;
        t.K_hi = (int64_t)khi;
        t.B_per_K = (int64_t)bpk;
        t.w_extra = (int64_t)wex;
        t.L = (int32_t)L;
        const Json *s0 = c.get("snr_lo"), *s1 = c.get("snr_hi");
        t.noiseless = !s0 || s0->kind == Json::kNull;
        t.snr_lo = t.noiseless ? 0.0 : s0->num;
        t.snr_hi = (!s1 || s1->kind != Json::kNum) ? INFINITY : s1->num;
        if (t.logN < 1 || t.logN > kMaxLogN || t.K_lo < 1 || t.K_hi < t.K_lo || t.B_per_K < 1 || t.B_per_K > 4096 ||
            t.w_extra < 0 || t.w_extra > 64 || t.L < 1 || t.L > kMaxL) {
            set_error("tuning cache: a class has values out of range");
            return SFFT_EINVAL;
        }
        out.push_back(t);
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_classes.swap(out);
    return SFFT_OK;
}

extern "C" void sfft_tuning_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_classes.clear();
}

extern "C" int32_t sfft_tuning_classes(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (int32_t)g_classes.size();
}
