// pp_types.h -- layouts shared by the host launcher and the kernels.
#pragma once
#include <cstdint>

#include "../../include/parparaw.h"

namespace pp {

// Parser tables in the form the kernels consume (built once by create).
struct Tables {
  uint8_t group_of[256];     // symbol -> group (Sec. 4.5 symbol groups)
  uint64_t trans[PP_MAX_GROUPS];       // byte s = next state of (group, s)
  uint64_t trans_run[PP_MAX_GROUPS];   // a catch-all run, then the group
  uint32_t emit[PP_MAX_GROUPS];        // bits [2s, 2s+1] = tag of (group, s)
  uint32_t rep[PP_MAX_SYMBOLS];        // symbol byte replicated into 4 lanes
  // Re-simulation step of one special symbol of group g read in state s,
  // after a run of catch-all symbols (r = 1) or directly (r = 0):
  // step[r][g][s] = next state | tag << 3 | kStepInv (the symbol's transition
  // enters the invalid state) | kStepSlow (r = 1 and the run is not all data
  // or enters the invalid state: re-simulated byte by byte).
  uint8_t step[2][PP_MAX_GROUPS][PP_MAX_STATES];
  uint8_t col_type[PP_MAX_COLUMNS];
  uint8_t str_slot[PP_MAX_COLUMNS];    // string column -> slot, else 0xFF
  uint8_t num_slot[PP_MAX_COLUMNS];    // numeric column -> slot, else 0xFF
  uint8_t num_states, num_groups, num_symbols, catch_all;
  uint8_t start_state, invalid_state, idempotent, num_columns;
  uint8_t num_str, num_num, partial, unit2;  // partial: more input follows; unit2: UTF-16LE code units
  uint32_t accept_mask;
  uint32_t skip_records;  // the first n records leave no row (Sec. 4.3)
};

struct Col {
  void* values;
  int64_t* offsets;
  uint8_t* validity;
  uint64_t values_cap;
};

// Per-parse scratch bookkeeping (device memory, zeroed by the init kernel).
struct Misc {
  unsigned long long first_invalid;  // atomicMin; ~0 = none
  uint32_t timeout;                  // a bounded wait expired
  uint32_t done;                     // the last tile wrote the totals below
  int64_t rows;                      // records emitted
  int32_t final_state;
  uint32_t pad;
  unsigned long long last_record_end;  // partial inputs: atomicMax of (last RD + 1)
  int64_t bytes_total[PP_MAX_STRING_COLUMNS];
  // inference (parparaw_infer): per field position the widest rank of the
  // chain int32 (1) < int64 (2) < float64 (3) < string (4); fields per record
  uint32_t inf_rank[PP_MAX_COLUMNS];
  uint32_t inf_min_fields, inf_max_fields;
};

// One input of a launch.
struct Job {
  const uint8_t* input;
  uint64_t len;
  uint64_t head;        // input address mod 16: tiles are 16-byte aligned
  uint64_t ntiles;
  uint64_t tile_base;   // first work item of this job
  uint64_t rows_cap;
  uint64_t bit_words;   // 32-bit words of each fail / null bitmap
  uint8_t* row_valid;
  pp_parse_result* result;
  uint32_t tables;      // index into the launch's table array
  uint32_t col0;        // index of column 0 in the launch's column array
  // scratch
  uint64_t* st_state;   // chain 1: per tile, flag | packed vector
  uint64_t* st_rc;      // chain 2: per tile, flag | records, column offset
  uint64_t* st_bytes;   // chain 3: per tile, per string slot, flag | byte count
  uint32_t* fail_bits;  // per row: rejected
  uint32_t* null_bits;  // per numeric slot, per row: empty or unconvertible
  Misc* misc;
};

// Kernel launch parameters.  A single parse carries its job, columns and
// tables inline (jobs == nullptr); a batch points at device arrays.
struct Launch {
  const Job* jobs;
  const Col* cols;
  const Tables* tables;
  uint32_t njobs;
  uint32_t first_item;  // the work queue's first item (0; testing: later, see PP_OPT_FIRST_ITEM)
  uint64_t total_tiles;
  unsigned long long* work_counter;
  uint64_t timeout_ns;
  unsigned long long* phase_cycles;  // profiling builds only; else nullptr
  Job job0;
  Tables tables0;
  Col cols0[PP_MAX_COLUMNS];
};

static_assert(sizeof(Job) % 8 == 0 && sizeof(Tables) % 4 == 0 && sizeof(Col) % 8 == 0,
              "descriptors are copied in 4- and 8-byte words");

constexpr uint8_t kStepInv = 0x20;
constexpr uint8_t kStepSlow = 0x40;

constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagInc = 2ull << 62;
constexpr uint64_t kFlagMask = 3ull << 62;

}  // namespace pp
