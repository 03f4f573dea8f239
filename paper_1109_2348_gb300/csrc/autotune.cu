// bwt_plan_autotune: picks the radix digit width and tile size for a plan by
// timing the real batch, and remembers the choice in a small JSON-lines file.
//
// Sweep: radix_bits in {8, 11, 16} x tile_keys in {1024, 2048, 4096} (16-bit
// digits are skipped if their scratch cannot be allocated), then the
// doubling rounds' digit width in {8, 10, 11} with the best of those; each
// candidate runs once untimed and then `repeats` times between CUDA events on
// the caller's stream; the fastest mean wins. The cache file holds one JSON
// object per line, with every candidate's mean time as
// [radix_bits, tile_keys, round_radix_bits (0 = by rank width), ms]:
//   {"gpu": "<device name>", "key": "<workload signature>", "radix_bits": 8,
//    "tile_keys": 4096, "round_radix_bits": 10, "ms": 1.234,
//    "candidates": [[8, 1024, 0, 1.5], ...]}
// The workload signature is the block count, total bytes, largest block and
// plan flags, so uneven batches of the same shape reuse one entry. A later
// entry for the same (gpu, key) overrides an earlier one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "bwt.h"
#include "plan_internal.h"

namespace {

std::string json_escape(const std::string& s) {
    std::string o;
    for (char c : s) {
        if (c == '"' || c == '\\') o.push_back('\\');
        o.push_back(c);
    }
    return o;
}

// value of "field": in one JSON line (string or integer/float token)
bool json_field(const std::string& line, const char* field, std::string* out) {
    const std::string pat = std::string("\"") + field + "\":";
    size_t p = line.find(pat);
    if (p == std::string::npos) return false;
    p += pat.size();
    while (p < line.size() && line[p] == ' ') ++p;
    if (p < line.size() && line[p] == '"') {
        std::string v;
        for (size_t q = p + 1; q < line.size(); ++q) {
            if (line[q] == '\\' && q + 1 < line.size()) {
                v.push_back(line[++q]);
            } else if (line[q] == '"') {
                *out = v;
                return true;
            } else {
                v.push_back(line[q]);
            }
        }
        return false;
    }
    size_t q = p;
    while (q < line.size() && line[q] != ',' && line[q] != '}') ++q;
    *out = line.substr(p, q - p);
    return true;
}

std::string gpu_name(int device) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
    return prop.name;
}

}  // namespace

extern "C" bwt_status bwt_plan_autotune(bwt_plan* plan, const uint8_t* d_in, const uint64_t* offsets,
                                        uint32_t num_blocks, uint8_t* d_L, int32_t* d_primary, void* stream,
                                        const char* cache_path, int repeats, int* out_radix_bits,
                                        int* out_tile_keys, float* out_ms) {
    if (!plan || !d_in || !offsets || !d_L || !d_primary || num_blocks == 0) return BWT_EINVAL;
    if (repeats < 1) repeats = 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(plan->device) != cudaSuccess) return BWT_ECUDA;
    // signature of the workload
    std::vector<uint64_t> off(num_blocks + 1);
    if (cudaMemcpy(off.data(), offsets, sizeof(uint64_t) * (num_blocks + 1), cudaMemcpyDefault) != cudaSuccess)
        return bwt::record_cuda(cudaGetLastError(), "cudaMemcpy offsets");
    uint64_t max_n = 0;
    for (uint32_t b = 0; b < num_blocks; ++b) max_n = std::max<uint64_t>(max_n, off[b + 1] - off[b]);
    std::ostringstream ks;
    ks << "blocks=" << num_blocks << ";bytes=" << off[num_blocks] << ";max_block=" << max_n
       << ";flags=" << plan->desc.flags;
    const std::string key = ks.str();
    const std::string gpu = gpu_name(plan->device);

    if (cache_path && *cache_path) {
        std::ifstream in(cache_path);
        std::string line, best_line;
        while (std::getline(in, line)) {
            std::string g, k;
            if (json_field(line, "gpu", &g) && json_field(line, "key", &k) && g == gpu && k == key) best_line = line;
        }
        std::string rb, tk, ms, rr;
        if (!best_line.empty() && json_field(best_line, "radix_bits", &rb) && json_field(best_line, "tile_keys", &tk)) {
            const int r = std::atoi(rb.c_str()), t = std::atoi(tk.c_str());
            const int rrb = json_field(best_line, "round_radix_bits", &rr) ? std::atoi(rr.c_str()) : 0;
            if (bwt_plan_set_radix(plan, r, t) == BWT_OK && bwt_plan_set_round_radix(plan, rrb) == BWT_OK) {
                if (out_radix_bits) *out_radix_bits = r;
                if (out_tile_keys) *out_tile_keys = t;
                if (out_ms) *out_ms = json_field(best_line, "ms", &ms) ? (float)std::atof(ms.c_str()) : 0.f;
                return BWT_OK;
            }
        }
    }

    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bwt::record_cuda(cudaGetLastError(), "cudaEventCreate");
    const int bits[] = {8, 11, 16};
    const int tiles[] = {1024, 2048, 4096};
    float best = 1e30f;
    int best_b = plan->rbits, best_t = plan->tile;
    bwt_status status = BWT_OK;
    std::ostringstream cand;  // every timed candidate, for the cache line
    auto add_cand = [&](int b, int t, int r, float ms) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "%s[%d, %d, %d, %.4f]", cand.tellp() > 0 ? ", " : "", b, t, r, ms);
        cand << buf;
    };
    for (int b : bits) {
        for (int t : tiles) {
            if ((status = bwt_plan_set_radix(plan, b, t)) != BWT_OK) {
                if (b == 16 && (status == BWT_ENOMEM || status == BWT_EINVAL)) {  // no room for its scratch
                    cudaGetLastError();
                    status = BWT_OK;
                    continue;
                }
                break;
            }
            if ((status = bwt_forward_batch(plan, d_in, offsets, num_blocks, d_L, d_primary, stream)) != BWT_OK) break;
            float total = 0.f;
            for (int r = 0; r < repeats && status == BWT_OK; ++r) {
                cudaEventRecord(e0, st);
                status = bwt_forward_batch(plan, d_in, offsets, num_blocks, d_L, d_primary, stream);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                if (status == BWT_OK) status = bwt_plan_last_status(plan);  // device-side status of the run
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                total += ms;
            }
            if (status != BWT_OK) break;
            const float mean = total / repeats;
            add_cand(b, t, plan->round_bits, mean);
            if (mean < best) {
                best = mean;
                best_b = b;
                best_t = t;
            }
        }
        if (status != BWT_OK) break;
    }
    // the doubling rounds' digit width, with the best first-sort choice
    int best_r = 0;
    if (status == BWT_OK) {
        bwt_plan_set_radix(plan, best_b, best_t);
        float best_round = 1e30f;
        for (int rbits : {8, 10, 11}) {
            if ((status = bwt_plan_set_round_radix(plan, rbits)) != BWT_OK) break;
            if ((status = bwt_forward_batch(plan, d_in, offsets, num_blocks, d_L, d_primary, stream)) != BWT_OK) break;
            float total = 0.f;
            for (int r = 0; r < repeats && status == BWT_OK; ++r) {
                cudaEventRecord(e0, st);
                status = bwt_forward_batch(plan, d_in, offsets, num_blocks, d_L, d_primary, stream);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                if (status == BWT_OK) status = bwt_plan_last_status(plan);  // device-side status of the run
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                total += ms;
            }
            if (status == BWT_OK) add_cand(best_b, best_t, rbits, total / repeats);
            if (status == BWT_OK && total / repeats < best_round) {
                best_round = total / repeats;
                best_r = rbits;
            }
        }
        if (best_round < best) best = best_round;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != BWT_OK) return status;
    bwt_plan_set_radix(plan, best_b, best_t);
    bwt_plan_set_round_radix(plan, best_r);
    // one run with the chosen configuration: outputs and statistics are its
    if ((status = bwt_forward_batch(plan, d_in, offsets, num_blocks, d_L, d_primary, stream)) != BWT_OK) return status;
    if ((status = bwt_plan_last_status(plan)) != BWT_OK) return status;
    if (out_radix_bits) *out_radix_bits = best_b;
    if (out_tile_keys) *out_tile_keys = best_t;
    if (out_ms) *out_ms = best;
    if (cache_path && *cache_path) {
        FILE* f = std::fopen(cache_path, "a");
        if (f) {
            std::fprintf(f,
                         "{\"gpu\": \"%s\", \"key\": \"%s\", \"radix_bits\": %d, \"tile_keys\": %d, "
                         "\"round_radix_bits\": %d, \"ms\": %.4f, \"candidates\": [%s]}\n",
                         json_escape(gpu).c_str(), json_escape(key).c_str(), best_b, best_t, best_r, best,
                         cand.str().c_str());
            std::fclose(f);
        }
    }
    return BWT_OK;
}
