// tune_cache.h -- the autotuner's cache file: a flat JSON object mapping
// string keys to integers, one entry per line,
//
//   {
//     "D3Q19/fp32/256x256x256/bgk/std/NVIDIA GB300/152": 16,
//     ...
//   }
//
// Host-only C++ (no CUDA), header-only so tests can build it with a plain
// C++ compiler.  Reading is tolerant: a missing or malformed file reads as
// empty, and entries it cannot parse are skipped.  Writing replaces the file
// through a temporary file and a rename, so a reader never sees half a file.
#pragma once
#include <cstdio>
#include <cstdlib>
#include <map>
#include <string>

#include <unistd.h>

namespace nlc {

// JSON string literal of s (quotes, backslashes and control bytes escaped)
inline std::string json_quote(const std::string& s) {
  std::string o = "\"";
  for (unsigned char c : s) {
    if (c == '"' || c == '\\') {
      o += '\\';
      o += (char)c;
    } else if (c < 0x20) {
      char b[8];
      std::snprintf(b, sizeof b, "\\u%04x", c);
      o += b;
    } else {
      o += (char)c;
    }
  }
  return o + "\"";
}

// Parses the flat object in text; returns false (and an empty map) on
// anything that is not such an object.
inline bool tune_cache_parse(const std::string& text, std::map<std::string, long>* out) {
  out->clear();
  size_t i = 0;
  const size_t n = text.size();
  auto ws = [&]() {
    while (i < n && (text[i] == ' ' || text[i] == '\n' || text[i] == '\r' || text[i] == '\t'))
      i++;
  };
  ws();
  if (i >= n || text[i] != '{') return false;
  i++;
  ws();
  if (i < n && text[i] == '}') return true;
  while (i < n) {
    ws();
    if (i >= n || text[i] != '"') break;
    i++;
    std::string key;
    bool ok = false;
    while (i < n) {
      const char c = text[i++];
      if (c == '"') {
        ok = true;
        break;
      }
      if (c == '\\') {
        if (i >= n) break;
        const char e = text[i++];
        if (e == 'u') {
          if (i + 4 > n) break;
          key += (char)std::strtol(text.substr(i, 4).c_str(), nullptr, 16);
          i += 4;
        } else if (e == 'n') {
          key += '\n';
        } else if (e == 't') {
          key += '\t';
        } else {
          key += e;
        }
      } else {
        key += c;
      }
    }
    if (!ok) break;
    ws();
    if (i >= n || text[i] != ':') break;
    i++;
    ws();
    const char* start = text.c_str() + i;
    char* end = nullptr;
    const long v = std::strtol(start, &end, 10);
    if (end == start) break;
    i += (size_t)(end - start);
    (*out)[key] = v;
    ws();
    if (i < n && text[i] == ',') {
      i++;
      continue;
    }
    if (i < n && text[i] == '}') return true;
    break;
  }
  out->clear();
  return false;
}

inline std::map<std::string, long> tune_cache_read(const std::string& path) {
  std::map<std::string, long> m;
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return m;
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
  std::fclose(f);
  tune_cache_parse(text, &m);
  return m;
}

// value of key in the cache at path; false if absent
inline bool tune_cache_get(const std::string& path, const std::string& key, long* value) {
  const std::map<std::string, long> m = tune_cache_read(path);
  auto it = m.find(key);
  if (it == m.end()) return false;
  *value = it->second;
  return true;
}

// sets key to value (keeping the other entries); false if the file cannot
// be written
inline bool tune_cache_put(const std::string& path, const std::string& key, long value) {
  std::map<std::string, long> m = tune_cache_read(path);
  m[key] = value;
  const std::string tmp = path + ".tmp." + std::to_string((long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  std::string text = "{\n";
  size_t k = 0;
  for (const auto& e : m) {
    text += "  " + json_quote(e.first) + ": " + std::to_string(e.second);
    text += ++k < m.size() ? ",\n" : "\n";
  }
  text += "}\n";
  const bool ok = std::fwrite(text.data(), 1, text.size(), f) == text.size();
  if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return false;
  }
  return true;
}

}  // namespace nlc
