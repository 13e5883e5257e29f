// Persisted autotuner choices.
//
// Both autotuners (the single-problem Euler planner and the batched kernel's
// ring and cluster shape) time candidates on the GPU the first time a shape is
// seen.  Their choices are kept in memory for the process and appended to a
// text file, one "key<TAB>value" line each, so that later processes on the same
// GPU model start with them.  The file is $CS_TUNE_CACHE when that variable is
// set (an empty value turns persistence off), else
// $XDG_CACHE_HOME/paper_2405_00366_gb300/tune.txt, else
// $HOME/.cache/paper_2405_00366_gb300/tune.txt.  A later line for the same key
// overrides an earlier one; lines that do not parse are ignored.  Keys carry
// the device's name, SM count and compute capability and a format version, so
// a file shared between machines only serves matching GPUs.  A stored choice is
// a preference, not a trusted input: the callers check it against the
// candidates they would time and re-tune when it matches none.
#include <sys/stat.h>

#include <algorithm>
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace cs {

namespace {

constexpr const char* kTuneFormat = "cs-tune-1";

struct TuneCache {
  std::mutex mu;
  bool loaded = false;
  std::string path;
  std::map<std::string, std::string> entries;
  long long tunings = 0;  // timed tuning runs in this process
  long long disk_hits = 0;
};

TuneCache& cache() {
  static TuneCache c;
  return c;
}

std::string default_path() {
  const char* env = std::getenv("CS_TUNE_CACHE");
  if (env) return std::string(env);
  const char* xdg = std::getenv("XDG_CACHE_HOME");
  if (xdg && *xdg) return std::string(xdg) + "/paper_2405_00366_gb300/tune.txt";
  const char* home = std::getenv("HOME");
  if (home && *home) return std::string(home) + "/.cache/paper_2405_00366_gb300/tune.txt";
  return std::string();
}

void make_parent_dirs(const std::string& path) {
  for (size_t i = 1; i < path.size(); ++i)
    if (path[i] == '/') {
      const std::string dir = path.substr(0, i);
      if (mkdir(dir.c_str(), 0755) != 0 && errno != EEXIST) return;
    }
}

void load_locked(TuneCache& c) {
  if (c.loaded) return;
  c.loaded = true;
  c.path = default_path();
  if (c.path.empty()) return;
  FILE* f = std::fopen(c.path.c_str(), "r");
  if (!f) return;
  char line[4096];
  while (std::fgets(line, sizeof line, f)) {
    std::string s(line);
    while (!s.empty() && (s.back() == '\n' || s.back() == '\r')) s.pop_back();
    const size_t tab = s.find('\t');
    if (tab == std::string::npos || tab == 0 || tab + 1 >= s.size()) continue;
    c.entries[s.substr(0, tab)] = s.substr(tab + 1);
  }
  std::fclose(f);
}

}  // namespace

std::string tune_device_tag(int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return std::string("unknown");
  std::string name(prop.name);
  for (char& ch : name)
    if (ch == '\t' || ch == '\n' || ch == '|') ch = ' ';
  return std::string(kTuneFormat) + "|" + name + "|sm" + std::to_string(prop.major) + std::to_string(prop.minor) +
         "|" + std::to_string(prop.multiProcessorCount);
}

bool tune_lookup(const std::string& key, std::string* value) {
  TuneCache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  load_locked(c);
  auto it = c.entries.find(key);
  if (it == c.entries.end()) return false;
  *value = it->second;
  return true;
}

void tune_store(const std::string& key, const std::string& value) {
  TuneCache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  load_locked(c);
  c.entries[key] = value;
  if (c.path.empty()) return;
  make_parent_dirs(c.path);
  FILE* f = std::fopen(c.path.c_str(), "a");
  if (!f) return;  // persistence is best effort: the choice stays in memory
  std::fprintf(f, "%s\t%s\n", key.c_str(), value.c_str());
  std::fclose(f);
}

void tune_note(bool timed) {
  TuneCache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  if (timed)
    ++c.tunings;
  else
    ++c.disk_hits;
}

}  // namespace cs

extern "C" cs_status cs_tune_info(int64_t* tunings, int64_t* disk_hits, char* path, int64_t path_len) {
  cs::TuneCache& c = cs::cache();
  std::lock_guard<std::mutex> lk(c.mu);
  cs::load_locked(c);
  if (tunings) *tunings = c.tunings;
  if (disk_hits) *disk_hits = c.disk_hits;
  if (path && path_len > 0) {
    const size_t n = std::min<size_t>(c.path.size(), (size_t)path_len - 1);
    c.path.copy(path, n);
    path[n] = '\0';
  }
  return CS_OK;
}
