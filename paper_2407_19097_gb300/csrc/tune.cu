// Tuned launch choices and their cache file (nrv_tune_load / nrv_tune_save).
//
// The render pass picks one of its variants, and the tensor-core convolution its row
// read-ahead and CTAs per SM, by timing the candidates on the real data at the first launch
// that needs the choice.  Every candidate computes the same result, so a choice changes only
// the time.  The choices live in one process-wide table keyed by a text description of what
// they depend on; the table can be written to a text file and read back by a later process,
// which then skips the timing.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace nrv {

namespace {
std::mutex g_mu;
std::map<std::string, int> g_table;
bool g_env_loaded = false;
uint64_t g_timed = 0;

nrv_status load_file(const char* path) {
    FILE* f = fopen(path, "r");
    if (!f) return fail(NRV_ERR_ARG, "cannot open tune cache %s", path);
    char line[512];
    int lineno = 0;
    nrv_status st = NRV_OK;
    while (fgets(line, sizeof(line), f)) {
        ++lineno;
        size_t len = strlen(line);
        while (len && (line[len - 1] == '\n' || line[len - 1] == '\r')) line[--len] = 0;
        if (len == 0 || line[0] == '#') continue;
        // "<key> = <value>", the key free text without '='
        char* eq = strrchr(line, '=');
        char* end = nullptr;
        const long v = eq ? strtol(eq + 1, &end, 10) : 0;
        if (!eq || end == eq + 1 || v < 0 || v > 0x7FFFFFFFL) {
            st = fail(NRV_ERR_ARG, "tune cache %s line %d: expected '<key> = <value>'", path, lineno);
            break;
        }
        std::string key(line, eq - line);
        while (!key.empty() && key.back() == ' ') key.pop_back();
        g_table[key] = (int)v;
    }
    fclose(f);
    return st;
}

void load_env_once() {
    if (g_env_loaded) return;
    g_env_loaded = true;
    const char* p = getenv("NRV_TUNE_CACHE");
    if (p && *p) {
        FILE* f = fopen(p, "r");
        if (f) {
            fclose(f);
            load_file(p);
            clear_error();
        }
    }
}
}  // namespace

bool tune_get(const std::string& key, int* value) {
    std::lock_guard<std::mutex> lock(g_mu);
    load_env_once();
    auto it = g_table.find(key);
    if (it == g_table.end()) return false;
    *value = it->second;
    return true;
}

void tune_put(const std::string& key, int value) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table[key] = value;
}

void tune_count_timing() {
    std::lock_guard<std::mutex> lock(g_mu);
    ++g_timed;
}

}  // namespace nrv

using namespace nrv;

extern "C" nrv_status nrv_tune_load(const char* path) {
    clear_error();
    if (!path) return fail(NRV_ERR_ARG, "null path");
    std::lock_guard<std::mutex> lock(g_mu);
    g_env_loaded = true;
    return load_file(path);
}

extern "C" nrv_status nrv_tune_save(const char* path) {
    clear_error();
    if (!path) return fail(NRV_ERR_ARG, "null path");
    std::lock_guard<std::mutex> lock(g_mu);
    FILE* f = fopen(path, "w");
    if (!f) return fail(NRV_ERR_ARG, "cannot write tune cache %s", path);
    fprintf(f, "# libnrv tuned launch choices: <key> = <value>\n");
    for (const auto& kv : g_table) fprintf(f, "%s = %d\n", kv.first.c_str(), kv.second);
    const bool ok = fclose(f) == 0;
    return ok ? NRV_OK : fail(NRV_ERR_ARG, "writing tune cache %s failed", path);
}

extern "C" int nrv_tune_count(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    load_env_once();
    return (int)g_table.size();
}

extern "C" uint64_t nrv_tune_timings(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    return g_timed;
}
