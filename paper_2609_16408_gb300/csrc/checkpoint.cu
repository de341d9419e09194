// Checkpoint file of rpa_energy_density (format in checkpoint.cuh).  Host code only.
#include "checkpoint.cuh"

#include <cerrno>
#include <cstring>

#include <sys/stat.h>
#include <unistd.h>

namespace rpa {

namespace {

constexpr char kMagic[8] = {'R', 'P', 'A', 'C', 'K', 'P', 'T', '1'};
constexpr long kHeaderBytes = 32;

struct Header {
  char magic[8];
  unsigned long long key;
  long long count;
  long long reserved;
};
static_assert(sizeof(Header) == kHeaderBytes, "header layout");

unsigned int record_check(const CkptRecord& r) {
  const unsigned long long h = fnv1a(kFnvBasis, &r, 20);
  return (unsigned int)(h ^ (h >> 32));
}

std::string errno_text() { return std::string(std::strerror(errno)); }

}  // namespace

unsigned long long fnv1a(unsigned long long h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

rpa_status Checkpoint::open(const std::string& path, unsigned long long key, long long count,
                            std::vector<CkptRecord>* recs, std::string* msg) {
  close();
  recs->clear();
  path_ = path;
  FILE* f = std::fopen(path.c_str(), "r+b");
  if (!f) {
    if (errno != ENOENT) {
      *msg = "checkpoint " + path + ": " + errno_text();
      return RPA_EINVAL;
    }
    f = std::fopen(path.c_str(), "w+b");
    if (!f) {
      *msg = "checkpoint " + path + ": cannot create: " + errno_text();
      return RPA_EINVAL;
    }
  }
  struct stat sb;
  if (fstat(fileno(f), &sb) != 0) {
    *msg = "checkpoint " + path + ": " + errno_text();
    std::fclose(f);
    return RPA_EINVAL;
  }
  long valid = kHeaderBytes;
  if (sb.st_size < kHeaderBytes) {
    // new (or cut inside its header, before any record): write the header
    Header h;
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.key = key;
    h.count = count;
    h.reserved = 0;
    if (ftruncate(fileno(f), 0) != 0 || std::fseek(f, 0, SEEK_SET) != 0 ||
        std::fwrite(&h, sizeof(h), 1, f) != 1 || std::fflush(f) != 0 ||
        fsync(fileno(f)) != 0) {
      *msg = "checkpoint " + path + ": cannot write the header: " + errno_text();
      std::fclose(f);
      return RPA_EINVAL;
    }
  } else {
    Header h;
    if (std::fseek(f, 0, SEEK_SET) != 0 || std::fread(&h, sizeof(h), 1, f) != 1) {
      *msg = "checkpoint " + path + ": cannot read the header";
      std::fclose(f);
      return RPA_EINVAL;
    }
    if (std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0) {
      *msg = "checkpoint " + path + ": not a checkpoint file of this library";
      std::fclose(f);
      return RPA_EINVAL;
    }
    if (h.key != key || h.count != count) {
      *msg = "checkpoint " + path +
             ": written for another problem (grid, inputs, frequencies, coarse set or options "
             "differ)";
      std::fclose(f);
      return RPA_EINVAL;
    }
    CkptRecord r;
    while (std::fread(&r, sizeof(r), 1, f) == 1) {
      if (r.entry < 0 || r.entry >= count || r.check != record_check(r)) break;
      recs->push_back(r);
      valid += (long)sizeof(r);
    }
    if (valid != (long)sb.st_size && ftruncate(fileno(f), valid) != 0) {
      *msg = "checkpoint " + path + ": cannot cut a partial record: " + errno_text();
      std::fclose(f);
      return RPA_EINVAL;
    }
  }
  if (std::fseek(f, valid, SEEK_SET) != 0) {
    *msg = "checkpoint " + path + ": " + errno_text();
    std::fclose(f);
    return RPA_EINVAL;
  }
  f_ = f;
  return RPA_OK;
}

rpa_status Checkpoint::append(std::vector<CkptRecord>& recs, std::string* msg) {
  if (!f_) {
    *msg = "checkpoint is not open";
    return RPA_EINVAL;
  }
  for (auto& r : recs) r.check = record_check(r);
  if (!recs.empty() &&
      (std::fwrite(recs.data(), sizeof(CkptRecord), recs.size(), f_) != recs.size() ||
       std::fflush(f_) != 0 || fsync(fileno(f_)) != 0)) {
    *msg = "checkpoint " + path_ + ": write failed: " + errno_text();
    return RPA_EINVAL;
  }
  return RPA_OK;
}

void Checkpoint::close() {
  if (f_) std::fclose(f_);
  f_ = nullptr;
}

}  // namespace rpa
