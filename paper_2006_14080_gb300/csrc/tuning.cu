// Persistent autotuning results: the tile configuration that
// mri_plan_autotune chose (coils per forward N tile, forward and adjoint
// operand stages), keyed by precision, problem shape and SM count, kept in a
// process-wide table that plans consult when they are created, and saved to
// or loaded from a small JSON file.  The configuration changes the schedule
// of the tensor-core products only, never their arithmetic, so a stale or
// foreign table can cost speed but never change a result.
#include <cctype>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "internal.h"

namespace mri {

namespace {

using Key = std::tuple<int, int, int, int, int, int>;  // precision, nx, ny, nk, nc, sms

std::mutex g_mu;
using Tiles = std::tuple<int, int, int>;  // forward coils per tile, forward stages, adjoint stages
std::map<Key, Tiles> g_table;

Key key_of(const mri_plan *p) { return Key(p->precision, p->nx, p->ny, p->nk, p->nc, p->num_sms); }

// Integer value of "name": <int> inside [b, e), or false.
bool find_int(const std::string &s, size_t b, size_t e, const char *name, long long *out) {
    const std::string pat = std::string("\"") + name + "\"";
    size_t q = s.find(pat, b);
    if (q == std::string::npos || q >= e) return false;
    q += pat.size();
    while (q < e && std::isspace((unsigned char)s[q])) ++q;
    if (q >= e || s[q] != ':') return false;
    ++q;
    while (q < e && std::isspace((unsigned char)s[q])) ++q;
    size_t r = q;
    if (r < e && s[r] == '-') ++r;
    if (r >= e || !std::isdigit((unsigned char)s[r])) return false;
    *out = std::strtoll(s.c_str() + q, nullptr, 10);
    return true;
}

}  // namespace

void tuning_record(const mri_plan *p) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table[key_of(p)] = Tiles(p->fwd_coils_per_tile, p->fwd_stages, p->adj_stages);
}

bool tuning_lookup(const mri_plan *p, int *fwd_coils_per_tile, int *fwd_stages, int *adj_stages) {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(key_of(p));
    if (it == g_table.end()) return false;
    *fwd_coils_per_tile = std::get<0>(it->second);
    *fwd_stages = std::get<1>(it->second);
    *adj_stages = std::get<2>(it->second);
    return true;
}

}  // namespace mri

using namespace mri;

extern "C" {

MRI_API int mri_tuning_save(const char *path) {
    if (!path) return set_error("null path"), MRI_ERR_INVALID;
    std::string text = "{\"format\": \"mrirecon-tuning\", \"version\": 1, \"entries\": [";
    {
        std::lock_guard<std::mutex> lock(g_mu);
        bool first = true;
        for (const auto &kv : g_table) {
            char buf[320];
            std::snprintf(buf, sizeof(buf),
                          "%s\n  {\"precision\": %d, \"nx\": %d, \"ny\": %d, \"nk\": %d, \"nc\": %d, \"sms\": %d, "
                          "\"fwd_coils_per_tile\": %d, \"fwd_stages\": %d, \"adj_stages\": %d}",
                          first ? "" : ",", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                          std::get<3>(kv.first), std::get<4>(kv.first), std::get<5>(kv.first),
                          std::get<0>(kv.second), std::get<1>(kv.second), std::get<2>(kv.second));
            text += buf;
            first = false;
        }
    }
    text += "\n]}\n";
    FILE *f = std::fopen(path, "w");
    if (!f) return set_error(std::string("cannot open ") + path + " for writing"), MRI_ERR_INVALID;
    const bool ok = std::fwrite(text.data(), 1, text.size(), f) == text.size();
    if (std::fclose(f) != 0 || !ok) return set_error(std::string("write to ") + path + " failed"), MRI_ERR_INVALID;
    return MRI_OK;
}

MRI_API int mri_tuning_load(const char *path) {
    if (!path) return set_error("null path"), MRI_ERR_INVALID;
    FILE *f = std::fopen(path, "r");
    if (!f) return set_error(std::string("cannot open ") + path), MRI_ERR_INVALID;
    std::string s;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, n);
    std::fclose(f);
    if (s.find("\"mrirecon-tuning\"") == std::string::npos)
        return set_error(std::string(path) + " is not a tuning file"), MRI_ERR_INVALID;
    const size_t list = s.find("\"entries\"");
    if (list == std::string::npos) return set_error("tuning file has no entries"), MRI_ERR_INVALID;
    std::map<Key, Tiles> parsed;
    size_t b = s.find('{', list);
    while (b != std::string::npos) {
        const size_t e = s.find('}', b);
        if (e == std::string::npos) return set_error("unterminated tuning entry"), MRI_ERR_INVALID;
        const char *names[] = {"precision", "nx",         "ny",         "nk",        "nc",
                               "sms",       "fwd_coils_per_tile", "fwd_stages", "adj_stages"};
        long long v[9];
        for (int q = 0; q < 9; ++q)
            if (!find_int(s, b, e, names[q], &v[q]))
                return set_error(std::string("tuning entry without integer \"") + names[q] + "\""), MRI_ERR_INVALID;
        if (v[6] < 1 || v[6] > 4)
            return set_error("tuning entry with coils per tile outside 1..4"), MRI_ERR_INVALID;
        for (int q = 7; q < 9; ++q)
            if (v[q] < 2 || v[q] > 4)
                return set_error("tuning entry with a stage count outside 2..4"), MRI_ERR_INVALID;
        parsed[Key((int)v[0], (int)v[1], (int)v[2], (int)v[3], (int)v[4], (int)v[5])] =
            Tiles((int)v[6], (int)v[7], (int)v[8]);
        b = s.find('{', e);
    }
    std::lock_guard<std::mutex> lock(g_mu);
    for (const auto &kv : parsed) g_table[kv.first] = kv.second;
    return MRI_OK;
}

MRI_API int mri_tuning_clear(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table.clear();
    return MRI_OK;
}

MRI_API int mri_tuning_count(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    return (int)g_table.size();
}

}  // extern "C"
