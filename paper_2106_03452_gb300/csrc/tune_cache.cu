// Persisted autotuner choices. With DPSR_TUNE_CACHE=<file> in the
// environment, every plane-path choice the autotuner makes is recorded in
// that file, and a later process on the same kind of device reads it back
// instead of timing the candidates again: the first solve of each r no longer
// carries the tuning time, and every process picks the same kernels (so the
// same inputs give the same rounding across runs).
//
// The file is JSON Lines, one choice per line:
//   {"cc": 103, "sms": 152, "driver": 13000, "r": 128, "kind": 3, "batch": 0, "path": 1, "ms": 0.0370}
// cc = compute capability x 10, sms = SM count, driver = CUDA driver version
// (the device key); r and kind (0 forward, 1 inverse, 2 backward forward,
// 3 adjoint plane pass) and batch (0 for a solo plan, else the instance count
// of a batch class) select the choice; path is 0 for the pencil passes, else
// the cluster size; ms is the time the choice was measured at (information
// only). Lines of other devices, and lines that do not parse, are kept as
// they are when the file is rewritten. The rewrite goes to a temporary file
// that then replaces the old one (rename is atomic on POSIX), so a reader
// never sees half a file; two processes tuning at once may each drop the
// other's newest line, which only costs a retune.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <unistd.h>

#include <mutex>
#include <string>
#include <vector>

namespace {

struct Entry {
  int cc, sms, driver, r, kind, batch, path;
  float ms;
};

std::mutex g_mu;
bool g_loaded = false;
std::vector<Entry> g_entries;      // this process's view of the file
std::vector<std::string> g_other;  // lines kept verbatim (other devices, unparsed)

const char* cache_path() {
  const char* p = getenv("DPSR_TUNE_CACHE");
  return p && *p ? p : nullptr;
}

bool device_key(int* cc, int* sms, int* driver) {
  int dev = 0, maj = 0, min = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDriverGetVersion(driver) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *cc = maj * 10 + min;
  return true;
}

bool parse(const char* line, Entry* e) {
  int n = 0;
  if (sscanf(line,
             " {\"cc\": %d, \"sms\": %d, \"driver\": %d, \"r\": %d, \"kind\": %d, \"batch\": %d, "
             "\"path\": %d, \"ms\": %f}%n",
             &e->cc, &e->sms, &e->driver, &e->r, &e->kind, &e->batch, &e->path, &e->ms, &n) != 8)
    return false;
  // 0 pencil passes, 1/2/4/8 cluster size, 3 the adjoint kind split by channel
  const bool valid_path = e->path == 0 || e->path == 1 || e->path == 2 || e->path == 3 || e->path == 4 || e->path == 8;
  return n > 0 && valid_path && e->kind >= 0 && e->kind < 4 && e->r >= 8 && e->batch >= 0;
}

// Reads the file once per process (caller holds g_mu).
void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = cache_path();
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char buf[512];
  while (fgets(buf, sizeof(buf), f)) {
    std::string s(buf);
    while (!s.empty() && (s.back() == '\n' || s.back() == '\r')) s.pop_back();
    if (s.empty()) continue;
    Entry e;
    if (parse(s.c_str(), &e)) {
      bool dup = false;  // a later line of the same key wins
      for (Entry& x : g_entries)
        if (x.cc == e.cc && x.sms == e.sms && x.driver == e.driver && x.r == e.r && x.kind == e.kind &&
            x.batch == e.batch) {
          x = e;
          dup = true;
        }
      if (!dup) g_entries.push_back(e);
    } else {
      g_other.push_back(s);
    }
  }
  fclose(f);
}

void save_locked() {
  const char* path = cache_path();
  if (!path) return;
  std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  bool ok = true;
  for (const std::string& s : g_other) ok = ok && fprintf(f, "%s\n", s.c_str()) >= 0;
  for (const Entry& e : g_entries)
    ok = ok && fprintf(f,
                       "{\"cc\": %d, \"sms\": %d, \"driver\": %d, \"r\": %d, \"kind\": %d, \"batch\": %d, "
                       "\"path\": %d, \"ms\": %.6f}\n",
                       e.cc, e.sms, e.driver, e.r, e.kind, e.batch, e.path, e.ms) >= 0;
  ok = (fclose(f) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path) != 0) remove(tmp.c_str());
}

}  // namespace

// The cached path of plane kind `kind` at grid size r for a solo plan
// (batch = 0) or a batch class of `batch` instances on the current device,
// or -1 when there is none (or no cache file is configured).
extern "C" int dpsr_internal_tc_lookup(int kind, int r, int batch) {
  if (!cache_path()) return -1;
  int cc, sms, driver;
  if (!device_key(&cc, &sms, &driver)) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  for (const Entry& e : g_entries)
    if (e.cc == cc && e.sms == sms && e.driver == driver && e.r == r && e.kind == kind && e.batch == batch)
      return e.path;
  return -1;
}

// Records a choice of the autotuner and rewrites the cache file.
extern "C" void dpsr_internal_tc_store(int kind, int r, int batch, int path, float ms) {
  if (!cache_path()) return;
  int cc, sms, driver;
  if (!device_key(&cc, &sms, &driver)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  const Entry n{cc, sms, driver, r, kind, batch, path, ms};
  bool found = false;
  for (Entry& e : g_entries)
    if (e.cc == cc && e.sms == sms && e.driver == driver && e.r == r && e.kind == kind && e.batch == batch) {
      e = n;
      found = true;
    }
  if (!found) g_entries.push_back(n);
  save_locked();
}
