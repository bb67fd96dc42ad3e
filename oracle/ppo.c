/*
 * ppo.c -- ParPaRaw ORACLE (test infrastructure only; see ppo.h).
 *
 * Plain sequential restatement of the method's result.  Every function names
 * the part of the paper it follows.  No blocking, no fusion, no reordering:
 * one byte at a time, left to right.
 *
 * Readings of the paper that this file fixes (the paper leaves them open):
 *   - tags come from a Mealy table emit[group][state] (Sec. 3.1 leaves the
 *     tagging rules format specific);
 *   - INV is absorbing and emits CONTROL; the first byte whose transition
 *     enters INV is reported (Sec. 4.3, "Validating format");
 *   - the trailing record (bytes after the last record delimiter) is emitted
 *     only if the final state is accepting; a trailing record delimiter does
 *     not open an empty record; empty input gives no rows;
 *   - a record whose field count differs from the schema, or with a numeric
 *     field that fails to convert, is rejected: its row is kept, every column
 *     is null, row_valid is 0 (Sec. 4.3, column-count validation);
 *   - an empty numeric field is null (Sec. 4.3, default values); an empty
 *     string field is a valid empty string;
 *   - a numeric slot holds the converted value of its field text when that
 *     text converts, and 0 otherwise (empty, failed, missing);
 *   - string bytes of present fields are stored even when the row is
 *     rejected (Arrow allows a null slot to span bytes);
 *   - string offsets are int64 (Arrow LargeUtf8).
 */
#define _GNU_SOURCE
#include "ppo.h"

#include <errno.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* ------------------------------------------------------------------ format */

int ppo_format_init(ppo_format* f, uint32_t S, uint32_t G, const uint8_t* next,
                    const uint8_t* emit, uint32_t nsym, const uint8_t* symbols,
                    const uint8_t* groups, uint8_t catch_all, uint8_t start_state,
                    uint8_t invalid_state, uint32_t accept_mask) {
  memset(f, 0, sizeof(*f));
  if (S == 0 || S > PPO_MAX_STATES || G == 0 || G > PPO_MAX_GROUPS) return -1;
  if (catch_all >= G || start_state >= S) return -1;
  if (invalid_state != PPO_NO_STATE && invalid_state >= S) return -1;
  f->num_states = S;
  f->num_groups = G;
  for (uint32_t g = 0; g < G; ++g)
    for (uint32_t s = 0; s < S; ++s) {
      if (next[g * S + s] >= S || emit[g * S + s] > PPO_CONTROL) return -1;
      f->next[g][s] = next[g * S + s];
      f->emit[g][s] = emit[g * S + s];
    }
  for (int b = 0; b < 256; ++b) f->group_of[b] = catch_all;
  for (uint32_t i = 0; i < nsym; ++i) {
    if (groups[i] >= G) return -1;
    f->group_of[symbols[i]] = groups[i];
  }
  f->start_state = start_state;
  f->invalid_state = invalid_state;
  f->accept_mask = accept_mask;
  f->catch_all = catch_all;
  f->unit = 1;
  return 0;
}

void ppo_format_set_utf16le(ppo_format* f) { f->unit = 2; }

/* ------------------------------------ Sec. 4.2: variable-length symbols */

static uint32_t unit16(const uint8_t* in, size_t i) { return (uint32_t)in[i] | ((uint32_t)in[i + 1] << 8); }
static int is_high(uint32_t u) { return u >= 0xD800 && u <= 0xDBFF; }
static int is_low(uint32_t u) { return u >= 0xDC00 && u <= 0xDFFF; }

/* Length in bytes and group of the symbol that starts at in[i]. */
static size_t symbol_at(const ppo_format* f, const uint8_t* in, size_t len, size_t i, uint8_t* group) {
  if (f->unit == 1) {
    *group = f->group_of[in[i]];
    return 1;
  }
  if (i + 2 > len) { /* a lone trailing byte: not a code unit, read as the catch-all */
    *group = f->catch_all;
    return 1;
  }
  const uint32_t u = unit16(in, i);
  if (is_high(u) && i + 4 <= len && is_low(unit16(in, i + 2))) {
    *group = f->catch_all; /* a code point beyond U+FFFF */
    return 4;
  }
  *group = u <= 0xFF ? f->group_of[u] : f->catch_all;
  return 2;
}

void ppo_state_vector_at(const ppo_format* f, const uint8_t* in, size_t len, size_t begin, size_t end,
                         uint8_t out[PPO_MAX_STATES]) {
  /* the chunk's first symbol: its first code unit, unless that unit is the
   * low half of a pair whose high half is the previous code unit */
  size_t first = begin;
  if (f->unit == 2 && begin >= 2 && begin + 2 <= len && is_low(unit16(in, begin)) &&
      is_high(unit16(in, begin - 2)))
    first = begin + 2;
  for (uint32_t i = 0; i < PPO_MAX_STATES; ++i) out[i] = (uint8_t)i;
  for (uint32_t i = 0; i < f->num_states; ++i) {
    uint8_t s = (uint8_t)i;
    for (size_t k = first; k < end;) {
      uint8_t g;
      k += symbol_at(f, in, len, k, &g);
      s = f->next[g][s];
    }
    out[i] = s;
  }
}

/* ------------------------------------------------- Sec. 3.1: vectors and o */

void ppo_state_vector(const ppo_format* f, const uint8_t* chunk, size_t len,
                      uint8_t out[PPO_MAX_STATES]) {
  /* one DFA instance per start state s_i, each run over the whole chunk */
  for (uint32_t i = 0; i < PPO_MAX_STATES; ++i) out[i] = (uint8_t)i;
  for (uint32_t i = 0; i < f->num_states; ++i) {
    uint8_t s = (uint8_t)i;
    for (size_t k = 0; k < len; ++k) s = f->next[f->group_of[chunk[k]]][s];
    out[i] = s;
  }
}

void ppo_compose(uint32_t S, const uint8_t* a, const uint8_t* b, uint8_t* out) {
  /* (a o b)_i = b_{a_i}: run the chunk of a, then the chunk of b */
  uint8_t tmp[PPO_MAX_STATES];
  for (uint32_t i = 0; i < S; ++i) tmp[i] = b[a[i]];
  memcpy(out, tmp, S);
}

void ppo_trace(const ppo_format* f, const uint8_t* in, size_t len, uint8_t* tags,
               uint8_t* states_after) {
  uint8_t s = f->start_state;
  for (size_t i = 0; i < len; ++i) {
    uint8_t g = f->group_of[in[i]];
    if (tags) tags[i] = f->emit[g][s];
    s = f->next[g][s];
    if (states_after) states_after[i] = s;
  }
}

/* ----------------------------------------------- Sec. 3.3: type conversion */

static int all_digits(const uint8_t* t, size_t n) {
  if (n == 0) return 0;
  for (size_t i = 0; i < n; ++i)
    if (t[i] < '0' || t[i] > '9') return 0;
  return 1;
}

static int two(const uint8_t* t) { return (t[0] - '0') * 10 + (t[1] - '0'); }
static int four(const uint8_t* t) { return two(t) * 100 + two(t + 2); }

/* calendar date + time of day -> seconds since the epoch, UTC, through the C
 * library's timegm; the date is rejected when timegm had to normalise it. */
static int civil_to_epoch(int Y, int M, int D, int h, int m, int s, int64_t* out) {
  if (Y < 1 || M < 1 || M > 12 || D < 1 || D > 31) return 0;
  if (h > 23 || m > 59 || s > 59) return 0;
  struct tm tm;
  memset(&tm, 0, sizeof(tm));
  tm.tm_year = Y - 1900;
  tm.tm_mon = M - 1;
  tm.tm_mday = D;
  tm.tm_hour = h;
  tm.tm_min = m;
  tm.tm_sec = s;
  time_t t = timegm(&tm);
  struct tm back;
  if (!gmtime_r(&t, &back)) return 0;
  if (back.tm_year != Y - 1900 || back.tm_mon != M - 1 || back.tm_mday != D) return 0;
  *out = (int64_t)t;
  return 1;
}

static int conv_int(const uint8_t* t, size_t n, int bits, int64_t* v) {
  char buf[PPO_NUMERIC_MAX_LEN + 1];
  size_t k = (n > 0 && t[0] == '-') ? 1 : 0;
  if (!all_digits(t + k, n - k)) return 0;
  memcpy(buf, t, n);
  buf[n] = 0;
  errno = 0;
  long long x = strtoll(buf, NULL, 10);
  if (errno == ERANGE) return 0;
  if (bits == 32 && (x < INT32_MIN || x > INT32_MAX)) return 0;
  *v = (int64_t)x;
  return 1;
}

static int conv_float(const uint8_t* t, size_t n, double* v) {
  /* syntax -?d+(.d+)? ; accepted while the decimal significand m < 2^53 and
   * the fraction has at most 22 digits (values that one correctly rounded
   * division m / 10^k represents exactly, Clinger's fast path). */
  size_t i = (n > 0 && t[0] == '-') ? 1 : 0;
  size_t int_start = i;
  while (i < n && t[i] >= '0' && t[i] <= '9') ++i;
  size_t int_len = i - int_start;
  size_t frac_len = 0;
  if (int_len == 0) return 0;
  if (i < n) {
    if (t[i] != '.') return 0;
    size_t fs = ++i;
    while (i < n && t[i] >= '0' && t[i] <= '9') ++i;
    frac_len = i - fs;
    if (frac_len == 0 || i != n) return 0;
  }
  if (frac_len > 22) return 0;
  uint64_t m = 0;
  for (size_t k = int_start; k < n; ++k) {
    if (t[k] == '.') continue;
    m = m * 10 + (uint64_t)(t[k] - '0');
    if (m >= (1ull << 53)) return 0;
  }
  char buf[PPO_NUMERIC_MAX_LEN + 1];
  memcpy(buf, t, n);
  buf[n] = 0;
  *v = strtod(buf, NULL);
  return 1;
}

static int conv_date(const uint8_t* t, size_t n, int32_t* v) {
  if (n != 10 || t[4] != '-' || t[7] != '-') return 0;
  if (!all_digits(t, 4) || !all_digits(t + 5, 2) || !all_digits(t + 8, 2)) return 0;
  int64_t e;
  if (!civil_to_epoch(four(t), two(t + 5), two(t + 8), 0, 0, 0, &e)) return 0;
  *v = (int32_t)(e / 86400);
  return 1;
}

static int conv_timestamp(const uint8_t* t, size_t n, int64_t* v) {
  if (n != 19 || t[4] != '-' || t[7] != '-' || (t[10] != ' ' && t[10] != 'T') ||
      t[13] != ':' || t[16] != ':')
    return 0;
  if (!all_digits(t, 4) || !all_digits(t + 5, 2) || !all_digits(t + 8, 2) ||
      !all_digits(t + 11, 2) || !all_digits(t + 14, 2) || !all_digits(t + 17, 2))
    return 0;
  return civil_to_epoch(four(t), two(t + 5), two(t + 8), two(t + 11), two(t + 14),
                        two(t + 17), v);
}

static int conv_clf(const uint8_t* t, size_t n, int64_t* v) {
  /* dd/Mon/yyyy:hh:mm:ss +hhmm (Common Log Format) */
  static const char* months[12] = {"Jan", "Feb", "Mar", "Apr", "May", "Jun",
                                   "Jul", "Aug", "Sep", "Oct", "Nov", "Dec"};
  if (n != 26 || t[2] != '/' || t[6] != '/' || t[11] != ':' || t[14] != ':' ||
      t[17] != ':' || t[20] != ' ' || (t[21] != '+' && t[21] != '-'))
    return 0;
  if (!all_digits(t, 2) || !all_digits(t + 7, 4) || !all_digits(t + 12, 2) ||
      !all_digits(t + 15, 2) || !all_digits(t + 18, 2) || !all_digits(t + 22, 4))
    return 0;
  int mon = 0;
  for (int k = 0; k < 12; ++k)
    if (memcmp(t + 3, months[k], 3) == 0) mon = k + 1;
  if (mon == 0) return 0;
  int oh = two(t + 22), om = two(t + 24);
  if (oh > 23 || om > 59) return 0;
  int64_t e;
  if (!civil_to_epoch(four(t + 7), mon, two(t), two(t + 12), two(t + 15), two(t + 18), &e))
    return 0;
  int64_t off = (int64_t)oh * 3600 + (int64_t)om * 60;
  *v = (t[21] == '+') ? e - off : e + off;
  return 1;
}

int ppo_convert(uint32_t type, const uint8_t* text, size_t len, void* out) {
  if (len == 0) {
    memset(out, 0, 8);
    return PPO_CONV_EMPTY;
  }
  memset(out, 0, 8);
  if (len > PPO_NUMERIC_MAX_LEN) return PPO_CONV_FAIL;
  int ok = 0;
  switch (type) {
    case PPO_INT32: {
      int64_t x;
      if ((ok = conv_int(text, len, 32, &x))) {
        int32_t y = (int32_t)x;
        memcpy(out, &y, 4);
      }
      break;
    }
    case PPO_INT64: {
      int64_t x;
      if ((ok = conv_int(text, len, 64, &x))) memcpy(out, &x, 8);
      break;
    }
    case PPO_FLOAT64: {
      double x;
      if ((ok = conv_float(text, len, &x))) memcpy(out, &x, 8);
      break;
    }
    case PPO_DATE_D: {
      int32_t x;
      if ((ok = conv_date(text, len, &x))) memcpy(out, &x, 4);
      break;
    }
    case PPO_TIMESTAMP_S: {
      int64_t x;
      if ((ok = conv_timestamp(text, len, &x))) memcpy(out, &x, 8);
      break;
    }
    case PPO_TIMESTAMP_CLF: {
      int64_t x;
      if ((ok = conv_clf(text, len, &x))) memcpy(out, &x, 8);
      break;
    }
    default:
      ok = 0;
  }
  if (!ok) memset(out, 0, 8);
  return ok ? PPO_CONV_OK : PPO_CONV_FAIL;
}

/* ------------------------------------------------- growable output buffers */

typedef struct {
  uint8_t* p;
  size_t n, cap;
} buf_t;

static void buf_reserve(buf_t* b, size_t need) {
  if (need <= b->cap) return;
  size_t c = b->cap ? b->cap : 64;
  while (c < need) c *= 2;
  b->p = (uint8_t*)realloc(b->p, c);
  b->cap = c;
}
static void buf_put(buf_t* b, const void* src, size_t n) {
  buf_reserve(b, b->n + n);
  memcpy(b->p + b->n, src, n);
  b->n += n;
}
static void buf_byte(buf_t* b, uint8_t v) { buf_put(b, &v, 1); }
static void bit_set(buf_t* b, int64_t i, int v) {
  size_t byte = (size_t)(i >> 3);
  if (byte >= b->n) {
    buf_reserve(b, byte + 1);
    memset(b->p + b->n, 0, byte + 1 - b->n);
    b->n = byte + 1;
  }
  if (v) b->p[byte] |= (uint8_t)(1u << (i & 7));
}

static int width_of(uint32_t type) {
  return (type == PPO_INT32 || type == PPO_DATE_D) ? 4 : 8;
}

/* --------------------------------------------- the sequential parse itself */

typedef struct {
  const ppo_format* f;
  const uint32_t* types;
  uint32_t C;
  buf_t values[PPO_MAX_COLUMNS];  /* string bytes, or fixed-width values */
  buf_t offsets[PPO_MAX_COLUMNS]; /* int64 offsets (string columns) */
  buf_t validity[PPO_MAX_COLUMNS];
  buf_t row_valid;
  int64_t bytes_total[PPO_MAX_COLUMNS];
  /* current record */
  uint32_t nfields;                              /* fields closed so far */
  uint8_t num[PPO_NUMERIC_MAX_LEN + 1];          /* data of the open numeric field */
  size_t num_len;
  int64_t field_end[PPO_MAX_COLUMNS];            /* string: end offset of field c */
  uint8_t field_conv[PPO_MAX_COLUMNS];           /* numeric: PPO_CONV_* of field c */
  uint64_t field_value[PPO_MAX_COLUMNS];
  int64_t rows, rejected;
  uint64_t skip, seen;                           /* records to skip (Sec. 4.3), records ended */
} parse_state;

static void on_data(parse_state* p, uint8_t b) {
  if (p->seen < p->skip) return; /* a skipped record keeps nothing */
  uint32_t c = p->nfields;
  if (c >= p->C) return; /* fields past the schema are dropped */
  if (p->types[c] == PPO_SKIP) return; /* a column that is not selected */
  if (p->types[c] == PPO_STRING) {
    buf_byte(&p->values[c], b);
    p->bytes_total[c] += 1;
  } else if (p->num_len <= PPO_NUMERIC_MAX_LEN) {
    p->num[p->num_len++] = b; /* length PPO_NUMERIC_MAX_LEN + 1 marks "too long" */
  }
}

static void end_field(parse_state* p) {
  uint32_t c = p->nfields;
  if (c < p->C && p->types[c] != PPO_SKIP && p->seen >= p->skip) {
    if (p->types[c] == PPO_STRING) {
      p->field_end[c] = (int64_t)p->values[c].n;
    } else {
      uint64_t v = 0;
      const uint8_t* text = p->num;
      size_t n = p->num_len;
      uint8_t narrow[PPO_NUMERIC_MAX_LEN + 1];
      int ok = 1;
      if (p->f->unit == 2 && n <= PPO_NUMERIC_MAX_LEN) { /* UTF-16LE text: ASCII code points only */
        ok = n % 2 == 0;
        for (size_t k = 0; ok && k < n / 2; ++k) {
          const uint32_t u = unit16(p->num, 2 * k);
          ok = u < 0x80;
          narrow[k] = (uint8_t)u;
        }
        text = narrow;
        n /= 2;
      }
      p->field_conv[c] = ok ? (uint8_t)ppo_convert(p->types[c], text, n, &v) : PPO_CONV_FAIL;
      p->field_value[c] = ok ? v : 0;
    }
  }
  p->num_len = 0;
  p->nfields += 1;
}

static void end_record(parse_state* p) {
  if (p->seen < p->skip) { /* Sec. 4.3, skipping records: it leaves no row */
    p->seen += 1;
    p->nfields = 0;
    p->num_len = 0;
    return;
  }
  p->seen += 1;
  int valid = (p->nfields == p->C);
  for (uint32_t c = 0; c < p->C; ++c)
    if (c < p->nfields && p->types[c] != PPO_STRING && p->types[c] != PPO_SKIP &&
        p->field_conv[c] == PPO_CONV_FAIL)
      valid = 0;
  for (uint32_t c = 0; c < p->C; ++c) {
    if (p->types[c] == PPO_SKIP) continue; /* nothing is stored for it */
    int present = c < p->nfields;
    int nonnull = 1;
    if (p->types[c] == PPO_STRING) {
      int64_t end = present ? p->field_end[c] : (int64_t)p->values[c].n;
      buf_put(&p->offsets[c], &end, 8);
    } else {
      uint64_t v = 0;
      if (present && p->field_conv[c] == PPO_CONV_OK) v = p->field_value[c];
      if (!present || p->field_conv[c] != PPO_CONV_OK) nonnull = 0;
      buf_put(&p->values[c], &v, (size_t)width_of(p->types[c]));
    }
    bit_set(&p->validity[c], p->rows, valid && nonnull);
  }
  bit_set(&p->row_valid, p->rows, valid);
  if (!valid) p->rejected += 1;
  p->rows += 1;
  p->nfields = 0;
  p->num_len = 0;
}

int ppo_parse(const ppo_format* f, const uint32_t* types, uint32_t C, const uint8_t* in,
              size_t len, ppo_result* out) {
  return ppo_parse_skip(f, types, C, in, len, 0, out);
}

int ppo_parse_skip(const ppo_format* f, const uint32_t* types, uint32_t C, const uint8_t* in,
                   size_t len, uint64_t skip_records, ppo_result* out) {
  memset(out, 0, sizeof(*out));
  if (C == 0 || C > PPO_MAX_COLUMNS) return -1;
  parse_state* p = (parse_state*)calloc(1, sizeof(parse_state));
  p->skip = skip_records;
  p->f = f;
  p->types = types;
  p->C = C;
  for (uint32_t c = 0; c < C; ++c)
    if (types[c] == PPO_STRING) {
      int64_t zero = 0;
      buf_put(&p->offsets[c], &zero, 8);
    }

  int64_t first_invalid = -1;
  size_t since_record = 0; /* bytes read since the last record delimiter */
  uint8_t s = f->start_state;
  for (size_t i = 0; i < len;) {
    uint8_t g;
    const size_t n = symbol_at(f, in, len, i, &g); /* one symbol (Sec. 4.2): n bytes */
    uint8_t tag = f->emit[g][s];
    uint8_t nxt = f->next[g][s];
    if (f->invalid_state != PPO_NO_STATE && nxt == f->invalid_state &&
        s != f->invalid_state && first_invalid < 0)
      first_invalid = (int64_t)i;
    switch (tag) {
      case PPO_DATA:
        for (size_t k = 0; k < n; ++k) on_data(p, in[i + k]);
        break;
      case PPO_FIELD: end_field(p); break;
      case PPO_RECORD: end_field(p); end_record(p); break;
      default: break; /* control symbol: not part of any field */
    }
    since_record = (tag == PPO_RECORD) ? 0 : since_record + n;
    s = nxt;
    i += n;
  }
  int accepting = (f->accept_mask >> s) & 1u;
  if (since_record > 0 && accepting) {
    end_field(p);
    end_record(p);
  }

  out->status = PPO_OK;
  if (first_invalid >= 0)
    out->status = PPO_E_INVALID_INPUT;
  else if (!accepting)
    out->status = PPO_E_UNTERMINATED;
  out->final_state = s;
  out->rows = p->rows;
  out->n_rejected = p->rejected;
  out->first_invalid_offset = first_invalid;
  out->num_columns = C;
  for (uint32_t c = 0; c < C; ++c) {
    out->types[c] = types[c];
    /* bitmaps cover every row even when the last bits are zero */
    bit_set(&p->validity[c], p->rows > 0 ? p->rows - 1 : 0, 0);
    out->values[c] = p->values[c].p ? p->values[c].p : calloc(1, 8);
    out->offsets[c] = (int64_t*)p->offsets[c].p;
    out->validity[c] = p->validity[c].p;
    out->bytes_total[c] = p->bytes_total[c];
  }
  bit_set(&p->row_valid, p->rows > 0 ? p->rows - 1 : 0, 0);
  out->row_valid = p->row_valid.p;
  free(p);
  return 0;
}

void ppo_free(ppo_result* r) {
  for (uint32_t c = 0; c < r->num_columns; ++c) {
    free(r->values[c]);
    free(r->offsets[c]);
    free(r->validity[c]);
  }
  free(r->row_valid);
  memset(r, 0, sizeof(*r));
}

/* ------------------------------------------- Sec. 4.3: type inference */

/* rank in the chain int32 < int64 < float64 < string of a field's narrowest type */
static int infer_rank(const uint8_t* text, size_t len) {
  uint8_t v[8];
  if (len <= PPO_NUMERIC_MAX_LEN) {
    if (ppo_convert(PPO_INT32, text, len, v) == PPO_CONV_OK) return 1;
    if (ppo_convert(PPO_INT64, text, len, v) == PPO_CONV_OK) return 2;
    if (ppo_convert(PPO_FLOAT64, text, len, v) == PPO_CONV_OK) return 3;
  }
  return 4;
}

int ppo_infer(const ppo_format* f, const uint8_t* in, size_t len, ppo_inference* out) {
  return ppo_infer_skip(f, in, len, 0, out);
}

int ppo_infer_skip(const ppo_format* f, const uint8_t* in, size_t len, uint64_t skip_records,
                   ppo_inference* out) {
  static const uint8_t type_of_rank[5] = {PPO_NO_TYPE, PPO_INT32, PPO_INT64, PPO_FLOAT64, PPO_STRING};
  int rank[PPO_MAX_COLUMNS] = {0};
  uint8_t text[PPO_NUMERIC_MAX_LEN + 1];
  size_t tlen = 0;       /* data bytes of the current field (only the first ones are kept) */
  uint32_t field = 0;    /* position of the current field in its record */
  uint64_t ended = 0;    /* records ended so far, skipped ones included */
  memset(out, 0, sizeof(*out));
  out->min_fields = 0xFFFFFFFFu;
  int64_t first_invalid = -1;
  size_t since_record = 0;
  uint8_t s = f->start_state;
  /* a field ends: its narrowest type widens its position's type */
  #define END_FIELD()                                                   \
    do {                                                                \
      if (ended >= skip_records && field < PPO_MAX_COLUMNS && tlen > 0) { \
        const int r = infer_rank(text, tlen);                           \
        if (r > rank[field]) rank[field] = r;                           \
      }                                                                 \
      tlen = 0;                                                         \
    } while (0)
  /* a record ends with field + 1 fields */
  #define END_RECORD()                                                  \
    do {                                                                \
      if (ended++ < skip_records) { field = 0; break; }                 \
      uint32_t n = field + 1 < PPO_INFER_MAX_FIELDS ? field + 1 : PPO_INFER_MAX_FIELDS; \
      if (n < out->min_fields) out->min_fields = n;                     \
      if (n > out->max_fields) out->max_fields = n;                     \
      out->records++;                                                   \
      field = 0;                                                        \
    } while (0)
  for (size_t i = 0; i < len; ++i) {
    const uint8_t g = f->group_of[in[i]];
    const uint8_t tag = f->emit[g][s];
    const uint8_t nxt = f->next[g][s];
    if (f->invalid_state != PPO_NO_STATE && nxt == f->invalid_state && s != f->invalid_state &&
        first_invalid < 0)
      first_invalid = (int64_t)i;
    switch (tag) {
      case PPO_DATA:
        if (tlen <= PPO_NUMERIC_MAX_LEN) text[tlen] = in[i];
        tlen++;
        break;
      case PPO_FIELD: END_FIELD(); field++; break;
      case PPO_RECORD: END_FIELD(); END_RECORD(); break;
      default: break;
    }
    since_record = (tag == PPO_RECORD) ? 0 : since_record + 1;
    s = nxt;
  }
  const int accepting = (f->accept_mask >> s) & 1u;
  if (since_record > 0 && accepting) {
    END_FIELD();
    END_RECORD();
  }
  #undef END_FIELD
  #undef END_RECORD
  if (out->records == 0) out->min_fields = 0;
  for (int c = 0; c < PPO_MAX_COLUMNS; ++c) out->type[c] = type_of_rank[rank[c]];
  out->status = PPO_OK;
  if (first_invalid >= 0)
    out->status = PPO_E_INVALID_INPUT;
  else if (!accepting)
    out->status = PPO_E_UNTERMINATED;
  out->first_invalid_offset = first_invalid;
  return 0;
}

/* Sec. 4.3, skipping rows: the pruning pass, one byte at a time.  `next`
 * walks the sorted list of skipped rows alongside the current row. */
size_t ppo_skip_rows(const uint8_t* in, size_t len, const uint64_t* rows, size_t nrows,
                     uint8_t terminator, uint8_t* out) {
  uint64_t row = 0;
  size_t next = 0, n = 0;
  for (size_t i = 0; i < len; ++i) {
    while (next < nrows && rows[next] < row) ++next;
    const int skipped = next < nrows && rows[next] == row;
    if (!skipped) out[n++] = in[i];
    if (in[i] == terminator) ++row;
  }
  return n;
}
