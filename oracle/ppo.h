/*
 * ppo.h -- ParPaRaw ORACLE (test infrastructure only).
 *
 * A plain, slow, obviously correct, sequential CPU restatement of what the
 * ParPaRaw method computes (Stehle & Jacobsen, "ParPaRaw: Massively Parallel
 * Parsing of Delimiter-Separated Raw Data"):
 *
 *   - a DFA over symbol groups drives the parse (Sec. 3.1, Table 1);
 *   - the per-chunk state-transition vector and its composite operator
 *     (Sec. 3.1) are given by their definitions, one DFA run per start state;
 *   - the parse itself is ONE left-to-right Mealy pass: the method reaches
 *     exactly the result of the sequential DFA run (Sec. 3.1), so the oracle
 *     is that run written out, byte by byte, with a 256-entry group table;
 *   - fields are gathered per column in record order (Sec. 3.3) into an
 *     Arrow-like layout (Sec. 5, Apache Arrow output);
 *   - type conversion (Sec. 3.3) uses the C library (strtoll, strtod, timegm)
 *     as its definition.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs may load or call this library.  It shares no code, header,
 * table or helper with the CUDA path, and imports nothing from it.
 */
#ifndef PPO_H
#define PPO_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPO_MAX_STATES 8
#define PPO_MAX_GROUPS 16
#define PPO_MAX_COLUMNS 64
#define PPO_NO_STATE 0xFF
#define PPO_NUMERIC_MAX_LEN 64

/* per-byte tags: the paper's three bitmap indexes (record delimiter, field
 * delimiter, control symbol) plus "part of the field" (Sec. 3.1). */
enum { PPO_DATA = 0, PPO_FIELD = 1, PPO_RECORD = 2, PPO_CONTROL = 3 };

enum {
  PPO_STRING = 0,
  PPO_INT32 = 1,
  PPO_INT64 = 2,
  PPO_FLOAT64 = 3,
  PPO_TIMESTAMP_S = 4,  /* YYYY-MM-DD[ T]hh:mm:ss -> int64 seconds, UTC */
  PPO_DATE_D = 5,       /* YYYY-MM-DD -> int32 days since 1970-01-01 */
  PPO_TIMESTAMP_CLF = 6, /* dd/Mon/yyyy:hh:mm:ss +hhmm -> int64 seconds, UTC */
  PPO_SKIP = 7           /* Sec. 4.3, selecting columns: the field counts, nothing is kept */
};

enum {
  PPO_OK = 0,
  PPO_E_INVALID_INPUT = -4,
  PPO_E_UNTERMINATED = -5
};

/* conversion outcomes */
enum { PPO_CONV_OK = 0, PPO_CONV_EMPTY = 1, PPO_CONV_FAIL = 2 };

typedef struct ppo_format {
  uint32_t num_states;                       /* S */
  uint32_t num_groups;                       /* G */
  uint8_t next[PPO_MAX_GROUPS][PPO_MAX_STATES]; /* transition table, one row per group */
  uint8_t emit[PPO_MAX_GROUPS][PPO_MAX_STATES]; /* tag emitted by (group, state) */
  uint8_t group_of[256];                     /* symbol -> group, catch-all elsewhere */
  uint8_t start_state;
  uint8_t invalid_state;                     /* PPO_NO_STATE if none */
  uint32_t accept_mask;                      /* bit s: state s accepting at end */
  uint8_t catch_all;                         /* group of every symbol not listed */
  uint8_t unit;                              /* Sec. 4.2: 1 = byte symbols; 2 = UTF-16LE */
} ppo_format;

typedef struct ppo_result {
  int32_t status;
  int32_t final_state;
  int64_t rows;
  int64_t n_rejected;
  int64_t first_invalid_offset;              /* -1 if the input never enters INV */
  uint32_t num_columns;
  uint32_t types[PPO_MAX_COLUMNS];
  /* STRING: values = bytes, offsets[rows+1]; others: values = rows fixed-width */
  void* values[PPO_MAX_COLUMNS];
  int64_t* offsets[PPO_MAX_COLUMNS];
  uint8_t* validity[PPO_MAX_COLUMNS];        /* Arrow bitmaps, LSB first */
  int64_t bytes_total[PPO_MAX_COLUMNS];      /* data bytes seen for a string column */
  uint8_t* row_valid;
} ppo_result;

/* Build a format from a transition table next[g*S+s], tag table emit[g*S+s]
 * and a symbol list; every byte not listed maps to catch_all. Returns 0 on
 * success, -1 on a malformed table. */
int ppo_format_init(ppo_format* f, uint32_t S, uint32_t G, const uint8_t* next,
                    const uint8_t* emit, uint32_t nsym, const uint8_t* symbols,
                    const uint8_t* groups, uint8_t catch_all, uint8_t start_state,
                    uint8_t invalid_state, uint32_t accept_mask);

/* Sec. 4.2, variable-length symbols: the format reads UTF-16LE code units
 * instead of bytes.  A symbol is a code unit, or a surrogate pair (a high
 * surrogate followed by a low one) read as one symbol; code points up to
 * U+00FF take the group that the byte of the same value has, every other one
 * the catch-all group.  A symbol's tag applies to all of its bytes; numeric
 * fields convert when every code point of their text is ASCII. */
void ppo_format_set_utf16le(ppo_format* f);

/* Sec. 4.2 with Sec. 3.1: the state-transition vector of the chunk
 * in[begin, end) of a whole input in[0, len): the DFA reads the symbols that
 * start in the chunk (the last one may end past it); a chunk whose first code
 * unit completes a surrogate pair begun in the previous chunk skips it. */
void ppo_state_vector_at(const ppo_format* f, const uint8_t* in, size_t len, size_t begin, size_t end,
                         uint8_t out[PPO_MAX_STATES]);

/* Sec. 3.1: state-transition vector of a chunk. out[i] = state reached after
 * reading the chunk when the DFA starts in state i (one DFA run per state). */
void ppo_state_vector(const ppo_format* f, const uint8_t* chunk, size_t len,
                      uint8_t out[PPO_MAX_STATES]);

/* Sec. 3.1: composite of two state-transition vectors, (a o b)_i = b[a_i]. */
void ppo_compose(uint32_t S, const uint8_t* a, const uint8_t* b, uint8_t* out);

/* The sequential run: per byte, the tag emitted and the state entered. */
void ppo_trace(const ppo_format* f, const uint8_t* in, size_t len, uint8_t* tags,
               uint8_t* states_after);

/* The full parse into Arrow-like columns (allocates; free with ppo_free). */
int ppo_parse(const ppo_format* f, const uint32_t* types, uint32_t num_columns,
              const uint8_t* in, size_t len, ppo_result* out);
void ppo_free(ppo_result* r);

/* The same parse with the first skip_records records skipped (Sec. 4.3,
 * skipping records): they are recognised but leave no row, no bytes, no
 * conversion and no reject; rows count from the next record. */
int ppo_parse_skip(const ppo_format* f, const uint32_t* types, uint32_t num_columns,
                   const uint8_t* in, size_t len, uint64_t skip_records, ppo_result* out);

/* Type conversion of one field's data bytes (Sec. 3.3). *out receives an
 * int32/int64/double bit pattern in its low bytes. Returns PPO_CONV_*. */
int ppo_convert(uint32_t type, const uint8_t* text, size_t len, void* out);

/* Sec. 4.3 (capabilities): column-count and numeric type inference.  The
 * records are those ppo_parse finds (same tags, same trailing-record rule).
 * min/max_fields: the fewest and the most fields of a record (a count
 * saturates at PPO_INFER_MAX_FIELDS; both 0 without records).  type[c]: the
 * widest, in the chain int32 < int64 < float64 < string, of the narrowest
 * types of the non-empty fields at position c (each field's narrowest type is
 * the first of int32, int64, float64 whose conversion accepts its text, else
 * string); PPO_NO_TYPE when position c holds no non-empty field. */
#define PPO_INFER_MAX_FIELDS 256
#define PPO_NO_TYPE 0xFF
typedef struct ppo_inference {
  int32_t status;
  uint32_t min_fields, max_fields;
  int64_t records;
  int64_t first_invalid_offset;
  uint8_t type[PPO_MAX_COLUMNS];
} ppo_inference;
int ppo_infer(const ppo_format* f, const uint8_t* in, size_t len, ppo_inference* out);

/* Sec. 4.3, skipping rows: a row is a physical line, its bytes up to and
 * including the next `terminator` byte (the last row may lack it), whatever
 * the quoting; rows count from 0.  Copies to out (capacity >= len) the bytes
 * of every row not listed in rows[0..nrows) (strictly increasing) and
 * returns how many it copied.  The parse then runs on what is left. */
size_t ppo_skip_rows(const uint8_t* in, size_t len, const uint64_t* rows, size_t nrows,
                     uint8_t terminator, uint8_t* out);
int ppo_infer_skip(const ppo_format* f, const uint8_t* in, size_t len, uint64_t skip_records,
                   ppo_inference* out);  /* ppo_infer over all but the first skip_records records */

#ifdef __cplusplus
}
#endif
#endif
