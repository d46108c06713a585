// Sequence ingest: FASTA / FASTQ text to residue codes, streaming, on the
// host (the data-format side of the paper's API, Sec. II.C.1).  A reader
// hands out batches of whole records as the (codes, offsets) arrays that
// dsa_db_load and dsa_align_batch take, plus names and header line numbers.
#include "dsa_internal.cuh"

#include <algorithm>
#include <cerrno>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

struct dsa_seqs {
  std::vector<uint8_t> codes;
  std::vector<uint64_t> offsets{0};
  std::string names;
  std::vector<uint64_t> name_off{0};
  std::vector<uint64_t> lines;
};

namespace {

constexpr uint8_t SKIP = 0xFE;   // whitespace inside a sequence line
constexpr uint8_t BAD = 0xFF;    // not a residue of the alphabet

}  // namespace

struct dsa_reader {
  // source: a file read in chunks, or a caller-owned memory buffer
  FILE* f = nullptr;
  const char* mem = nullptr;
  uint64_t mem_len = 0, mem_pos = 0;
  std::vector<char> buf;    // file bytes not yet consumed are buf[beg, end)
  size_t beg = 0, end = 0;
  size_t chunk = 4u << 20;
  bool src_done = false;    // no more bytes to read from the source
  uint64_t line_no = 0;     // lines handed out so far
  uint8_t table[256];
  uint32_t flags = 0;
  // a header line read ahead (the next record's), or a whole record that did
  // not fit the previous batch
  bool have_header = false;
  std::string header;
  uint64_t header_line = 0;
  bool have_pending = false;
  std::vector<uint8_t> pend_codes;
  std::string pend_name;
  uint64_t pend_line = 0;
  int err = DSA_OK;         // sticky error
  std::string err_msg;
};

namespace {

void build_table(dsa_reader* r, int alphabet) {
  memset(r->table, BAD, sizeof r->table);
  for (const char c : {' ', '\t', '\r', '\v', '\f'}) r->table[(uint8_t)c] = SKIP;
  auto set = [&](char c, uint8_t code) {
    r->table[(uint8_t)c] = code;
    if (c >= 'A' && c <= 'Z') r->table[(uint8_t)(c - 'A' + 'a')] = code;
  };
  uint8_t unknown = 0;
  if (alphabet == DSA_ALPHABET_DNA4 || alphabet == DSA_ALPHABET_DNA5) {
    const char* letters = "ACGT";
    for (int k = 0; k < 4; ++k) set(letters[k], (uint8_t)k);
    set('U', 3);
    if (alphabet == DSA_ALPHABET_DNA5) {
      set('N', 4);
      for (const char c : {'R', 'Y', 'S', 'W', 'K', 'M', 'B', 'D', 'H', 'V'}) set(c, 4);
      unknown = 4;
    }
  } else {
    const char* letters = "ARNDCQEGHILKMFPSTWYVBZX*";
    for (int k = 0; letters[k]; ++k) set(letters[k], (uint8_t)k);
    for (const char c : {'U', 'O', 'J'}) set(c, 22);   // X
    unknown = 22;
  }
  if (r->flags & DSA_READ_MAP_UNKNOWN) {
    for (int c = 33; c < 127; ++c)   // printable, not a space
      if (r->table[c] == BAD && c != '>' && c != '@') r->table[c] = unknown;
  }
}

// Next line of the source without its "\n" (and a "\r" before it); the view
// stays valid until the next call.  Returns false at the end of the input.
bool next_line(dsa_reader* r, const char*& p, size_t& n) {
  if (r->mem) {
    if (r->mem_pos >= r->mem_len) return false;
    const char* s = r->mem + r->mem_pos;
    const size_t left = (size_t)(r->mem_len - r->mem_pos);
    const char* nl = static_cast<const char*>(memchr(s, '\n', left));
    const size_t len = nl ? (size_t)(nl - s) : left;
    r->mem_pos += len + (nl ? 1 : 0);
    p = s;
    n = len;
  } else {
    for (;;) {
      const char* s = r->buf.data() + r->beg;
      const char* nl = static_cast<const char*>(memchr(s, '\n', r->end - r->beg));
      if (nl) {
        p = s;
        n = (size_t)(nl - s);
        r->beg += n + 1;
        break;
      }
      if (r->src_done) {
        if (r->beg == r->end) return false;
        p = s;   // last line without a newline
        n = r->end - r->beg;
        r->beg = r->end;
        break;
      }
      // move the partial line to the front, grow if it fills the buffer, refill
      if (r->beg > 0) {
        memmove(r->buf.data(), r->buf.data() + r->beg, r->end - r->beg);
        r->end -= r->beg;
        r->beg = 0;
      }
      if (r->end == r->buf.size()) r->buf.resize(r->buf.size() * 2);
      const size_t got = fread(r->buf.data() + r->end, 1, r->buf.size() - r->end, r->f);
      r->end += got;
      if (got == 0) r->src_done = true;
    }
  }
  if (n > 0 && p[n - 1] == '\r') --n;
  ++r->line_no;
  return true;
}

bool blank(const char* p, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (p[k] != ' ' && p[k] != '\t' && p[k] != '\v' && p[k] != '\f') return false;
  return true;
}

int fail(dsa_reader* r, int code, const std::string& msg) {
  r->err = code;
  r->err_msg = msg;
  dsa::set_error("%s", msg.c_str());
  return code;
}

// Residues of one sequence line appended to `out`.
int encode_line(dsa_reader* r, const char* p, size_t n, std::vector<uint8_t>& out) {
  const size_t at = out.size();
  out.resize(at + n);
  uint8_t* o = out.data() + at;
  size_t w = 0;
  for (size_t k = 0; k < n; ++k) {
    const uint8_t c = r->table[(uint8_t)p[k]];
    if (c < SKIP) {
      o[w++] = c;
    } else if (c == BAD) {
      out.resize(at);
      char ch[8];
      if (p[k] >= 33 && p[k] < 127) snprintf(ch, sizeof ch, "'%c'", p[k]);
      else snprintf(ch, sizeof ch, "0x%02x", (unsigned)(uint8_t)p[k]);
      return fail(r, DSA_ERR_INVALID_ARG, "line " + std::to_string(r->line_no) + ": character " +
                                              ch + " is not a residue of the alphabet");
    }
  }
  out.resize(at + w);
  return DSA_OK;
}

// One record (its header already in r->header) into codes/name.  The next
// record's header, if one was read, is left in r->header.
int read_record(dsa_reader* r, std::vector<uint8_t>& codes, std::string& name, uint64_t& line) {
  const char kind = r->header[0];
  name.assign(r->header, 1, std::string::npos);
  line = r->header_line;
  r->have_header = false;
  const char* p;
  size_t n;
  if (kind == '>') {
    while (next_line(r, p, n)) {
      if (n > 0 && (p[0] == '>' || p[0] == '@')) {
        r->header.assign(p, n);
        r->header_line = r->line_no;
        r->have_header = true;
        return DSA_OK;
      }
      if (n > 0 && p[0] == ';') continue;   // comment line
      if (int rc = encode_line(r, p, n, codes)) return rc;
    }
    return DSA_OK;
  }
  // FASTQ: sequence lines up to the '+' line, then as many quality
  // characters as residues
  const size_t start = codes.size();
  bool plus = false;
  while (next_line(r, p, n)) {
    if (n > 0 && p[0] == '+') {
      plus = true;
      break;
    }
    if (int rc = encode_line(r, p, n, codes)) return rc;
  }
  if (!plus)
    return fail(r, DSA_ERR_INVALID_ARG, "line " + std::to_string(line) +
                                            ": FASTQ record has no '+' line");
  const uint64_t want = codes.size() - start;
  uint64_t have = 0;
  while (have < want) {
    if (!next_line(r, p, n))
      return fail(r, DSA_ERR_INVALID_ARG, "line " + std::to_string(line) +
                                              ": FASTQ quality shorter than the sequence");
    for (size_t k = 0; k < n; ++k)
      if (p[k] != ' ' && p[k] != '\t') ++have;
  }
  if (have != want)
    return fail(r, DSA_ERR_INVALID_ARG, "line " + std::to_string(r->line_no) +
                                            ": FASTQ quality longer than the sequence");
  return DSA_OK;
}

// Reads up to the next record's header; false at the end of the input.
int find_header(dsa_reader* r, bool& found) {
  found = r->have_header;
  if (found) return DSA_OK;
  const char* p;
  size_t n;
  while (next_line(r, p, n)) {
    if (blank(p, n)) continue;
    if (p[0] != '>' && p[0] != '@')
      return fail(r, DSA_ERR_INVALID_ARG, "line " + std::to_string(r->line_no) +
                                              ": a record must start with '>' or '@'");
    r->header.assign(p, n);
    r->header_line = r->line_no;
    r->have_header = found = true;
    return DSA_OK;
  }
  return DSA_OK;
}

int open_common(int alphabet, uint32_t flags, dsa_reader** out, dsa_reader*& r) {
  if (!out) { dsa::set_error("dsa_reader_open: NULL argument"); return DSA_ERR_INVALID_ARG; }
  *out = nullptr;
  if (alphabet != DSA_ALPHABET_DNA4 && alphabet != DSA_ALPHABET_DNA5 &&
      alphabet != DSA_ALPHABET_PROTEIN) {
    dsa::set_error("unknown alphabet %d", alphabet);
    return DSA_ERR_INVALID_ARG;
  }
  if (flags & ~(DSA_READ_MAP_UNKNOWN | DSA_READ_SKIP_EMPTY)) {
    dsa::set_error("unknown reader flags 0x%x", flags);
    return DSA_ERR_INVALID_ARG;
  }
  r = new (std::nothrow) dsa_reader;
  if (!r) { dsa::set_error("host allocation failed"); return DSA_ERR_OOM; }
  r->flags = flags;
  build_table(r, alphabet);
  return DSA_OK;
}

}  // namespace

extern "C" int dsa_reader_open(const char* path, int alphabet, uint32_t flags, uint64_t chunk_bytes,
                               dsa_reader** out) {
  if (!path) { dsa::set_error("dsa_reader_open: NULL path"); return DSA_ERR_INVALID_ARG; }
  dsa_reader* r = nullptr;
  DSA_TRY(open_common(alphabet, flags, out, r));
  r->f = fopen(path, "rb");
  if (!r->f) {
    dsa::set_error("cannot open %s: %s", path, strerror(errno));
    delete r;
    return DSA_ERR_INVALID_ARG;
  }
  if (chunk_bytes) r->chunk = (size_t)std::max<uint64_t>(chunk_bytes, 16);
  try {
    r->buf.resize(r->chunk);
  } catch (...) {
    fclose(r->f);
    delete r;
    dsa::set_error("host allocation failed");
    return DSA_ERR_OOM;
  }
  *out = r;
  return DSA_OK;
}

extern "C" int dsa_reader_open_mem(const char* data, uint64_t len, int alphabet, uint32_t flags,
                                   dsa_reader** out) {
  if (!data && len) { dsa::set_error("dsa_reader_open_mem: NULL data"); return DSA_ERR_INVALID_ARG; }
  dsa_reader* r = nullptr;
  DSA_TRY(open_common(alphabet, flags, out, r));
  r->mem = data ? data : "";
  r->mem_len = len;
  *out = r;
  return DSA_OK;
}

extern "C" int dsa_reader_next(dsa_reader* r, uint64_t max_residues, uint32_t max_seqs,
                               dsa_seqs** out) {
  if (!r || !out) { dsa::set_error("dsa_reader_next: NULL argument"); return DSA_ERR_INVALID_ARG; }
  *out = nullptr;
  if (r->err) {
    dsa::set_error("%s", r->err_msg.c_str());
    return r->err;
  }
  if (max_seqs == 0 || max_seqs == UINT32_MAX) max_seqs = UINT32_MAX - 1;
  dsa_seqs* s = new (std::nothrow) dsa_seqs;
  if (!s) { dsa::set_error("host allocation failed"); return DSA_ERR_OOM; }
  try {
    const bool skip_empty = r->flags & DSA_READ_SKIP_EMPTY;
    auto add = [&](const std::string& name, uint64_t line) {   // close the record ending here
      s->offsets.push_back(s->codes.size());
      s->names += name;
      s->name_off.push_back(s->names.size());
      s->lines.push_back(line);
    };
    if (r->have_pending) {   // the record that did not fit the last batch
      r->have_pending = false;
      s->codes.swap(r->pend_codes);
      r->pend_codes.clear();
      add(r->pend_name, r->pend_line);
    }
    std::string name;
    uint64_t line = 0;
    while (s->lines.size() < max_seqs) {
      bool found = false;
      if (int rc = find_header(r, found)) { delete s; return rc; }
      if (!found) break;
      const size_t from = s->codes.size();
      if (int rc = read_record(r, s->codes, name, line)) { delete s; return rc; }
      const size_t len = s->codes.size() - from;
      if (len == 0 && skip_empty) continue;
      if (max_residues && !s->lines.empty() && s->codes.size() > max_residues) {
        // does not fit: keep it for the next batch
        r->pend_codes.assign(s->codes.begin() + from, s->codes.end());
        s->codes.resize(from);
        r->pend_name = name;
        r->pend_line = line;
        r->have_pending = true;
        break;
      }
      add(name, line);
      if (max_residues && s->codes.size() >= max_residues) break;
    }
  } catch (const std::bad_alloc&) {
    delete s;
    return fail(r, DSA_ERR_OOM, "host allocation failed");
  }
  if (s->lines.empty()) {
    delete s;
    return DSA_OK;   // end of input
  }
  *out = s;
  return DSA_OK;
}

extern "C" int dsa_reader_close(dsa_reader* r) {
  if (!r) return DSA_OK;
  if (r->f) fclose(r->f);
  delete r;
  return DSA_OK;
}

extern "C" int dsa_seqs_get(const dsa_seqs* s, const uint8_t** codes, const uint64_t** offsets,
                            uint32_t* n_seqs, const char** names, const uint64_t** name_offsets,
                            const uint64_t** lines) {
  if (!s) { dsa::set_error("dsa_seqs_get: NULL batch"); return DSA_ERR_INVALID_ARG; }
  if (codes) *codes = s->codes.data();
  if (offsets) *offsets = s->offsets.data();
  if (n_seqs) *n_seqs = (uint32_t)s->lines.size();
  if (names) *names = s->names.data();
  if (name_offsets) *name_offsets = s->name_off.data();
  if (lines) *lines = s->lines.data();
  return DSA_OK;
}

extern "C" int dsa_seqs_free(dsa_seqs* s) {
  delete s;
  return DSA_OK;
}
