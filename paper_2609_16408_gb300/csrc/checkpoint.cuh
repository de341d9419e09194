// Checkpoint file of rpa_energy_density: the finished (frequency, coarse point) entries of
// d on C_g, appended as they complete, so that a run of many hours that stops (a killed job,
// a node failure) resumes with only the unfinished entries.  Host code only.
//
// Layout (little-endian as written by the host): a 32-byte header
//   magic "RPACKPT1" | key (u64, fingerprint of the problem) | count (i64, nw x P entries) |
//   reserved (i64, 0)
// followed by 24-byte records
//   entry (i64, k P + j: frequency k, coarse point j) | d (f64) | status (i32, the rpa_status
//   of the block that computed it: RPA_OK, RPA_ENOCONV or RPA_EBREAKDOWN) | check (u32,
//   fingerprint of the first 20 bytes).
// A record whose check fails, whose entry is out of range, or which is cut short ends the
// valid part of the file; the file is truncated there before new records are appended.
#pragma once
#include <cstdio>
#include <string>
#include <vector>

#include "rpa.h"

namespace rpa {

struct CkptRecord {
  long long entry;
  double d;
  int status;
  unsigned int check;
};
static_assert(sizeof(CkptRecord) == 24, "record layout");

// 64-bit FNV-1a over n bytes, continuing from h
unsigned long long fnv1a(unsigned long long h, const void* p, size_t n);
constexpr unsigned long long kFnvBasis = 1469598103934665603ull;

class Checkpoint {
 public:
  Checkpoint() = default;
  Checkpoint(const Checkpoint&) = delete;
  Checkpoint& operator=(const Checkpoint&) = delete;
  ~Checkpoint() { close(); }
  // Opens (or creates) the file.  An existing file must carry the same key and count
  // (RPA_EINVAL otherwise, with the reason in *msg); its valid records are returned in
  // *recs and it is reopened for appending after them.  RPA_EINVAL also for a file that
  // cannot be opened or written.
  rpa_status open(const std::string& path, unsigned long long key, long long count,
                  std::vector<CkptRecord>* recs, std::string* msg);
  // Appends records (their check fields are filled in) and flushes them to the device.
  rpa_status append(std::vector<CkptRecord>& recs, std::string* msg);
  void close();

 private:
  FILE* f_ = nullptr;
  std::string path_;
};

}  // namespace rpa
