// Process-wide tuning table: shape key -> chosen launch / tile variant, with a flat JSON file
// format {"key": choice, ...} for persistence between processes.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "cs_internal.h"

namespace cs {
namespace {
std::mutex g_mu;
std::map<std::string, int>& table() {
  static std::map<std::string, int> t;
  return t;
}
}  // namespace

bool tune_lookup(const std::string& key, int* choice) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = table().find(key);
  if (it == table().end()) return false;
  *choice = it->second;
  return true;
}

void tune_store(const std::string& key, int choice) {
  std::lock_guard<std::mutex> lk(g_mu);
  table()[key] = choice;
}

}  // namespace cs

extern "C" int cs_tune_save(const char* path) {
  if (!path) return cs::set_error(CS_EINVAL, "cs_tune_save: null path");
  std::lock_guard<std::mutex> lk(cs::g_mu);
  FILE* f = fopen(path, "w");
  if (!f) return cs::set_error(CS_EINVAL, "cs_tune_save: cannot open %s", path);
  fprintf(f, "{");
  bool first = true;
  for (const auto& kv : cs::table()) {
    fprintf(f, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
    first = false;
  }
  fprintf(f, "\n}\n");
  fclose(f);
  return CS_OK;
}

extern "C" int cs_tune_load(const char* path) {
  if (!path) return cs::set_error(CS_EINVAL, "cs_tune_load: null path");
  FILE* f = fopen(path, "r");
  if (!f) return cs::set_error(CS_EINVAL, "cs_tune_load: cannot open %s", path);
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
  fclose(f);
  // Accepts exactly the flat object written by cs_tune_save: "key": integer pairs.
  size_t pos = 0;
  int loaded = 0;
  while (true) {
    size_t q0 = text.find('"', pos);
    if (q0 == std::string::npos) break;
    size_t q1 = text.find('"', q0 + 1);
    if (q1 == std::string::npos) return cs::set_error(CS_EINVAL, "cs_tune_load: malformed key");
    size_t colon = text.find(':', q1);
    if (colon == std::string::npos) return cs::set_error(CS_EINVAL, "cs_tune_load: missing ':'");
    char* end = nullptr;
    long v = strtol(text.c_str() + colon + 1, &end, 10);
    if (end == text.c_str() + colon + 1) return cs::set_error(CS_EINVAL, "cs_tune_load: bad value");
    cs::tune_store(text.substr(q0 + 1, q1 - q0 - 1), static_cast<int>(v));
    ++loaded;
    pos = static_cast<size_t>(end - text.c_str());
  }
  (void)loaded;
  return CS_OK;
}
