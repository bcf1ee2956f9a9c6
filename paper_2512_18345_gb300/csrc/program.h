// Stage programs: the key-switching pipeline of a list of items (key
// switches, rotations, relinearisations, hoisted ModUp / ModDown halves),
// emitted stage by stage so that one launch processes the same stage of every
// item (Section IV-A multi-polynomial caching and batching: B sequences per
// stage instead of one).
#pragma once
#include <vector>

#include "ctx.h"

// IT_IPX: the inner product of a shared ModUp (slot ext_slot, read through sigma_galois) left in
// the extended basis: out [2][level+K][N] = u, plus P sigma(in2) on the q-limbs of u_0 when in2 is
// given (double hoisting keeps the rotation in Q_l u P).  IT_MDX: ModDown alone of `npoly`
// extended-basis polynomials in [npoly][level+K][N] to out [npoly][level][N].
enum ItemKind { IT_KS = 0, IT_ROTATE = 1, IT_RELIN = 2, IT_MODUP = 3, IT_MODDOWN = 4, IT_IPX = 5, IT_MDX = 6 };

struct Item {
  int kind = IT_KS;
  int level = 0;
  uint32_t galois = 1;             // rotation Galois element (1: none)
  const uint32_t *in = nullptr;    // KS / MODUP: d [level][N]; ROTATE / MODDOWN: ct [2][level][N]; RELIN: a;
                                   // IPX: the polynomial that was ModUp'ed [level][N]; MDX: [npoly][level+K][N]
  const uint32_t *in2 = nullptr;   // RELIN: b; IPX: pass-through c0 [level][N] or null
  uint32_t *out = nullptr;         // [2][level][N] (not for MODUP)
  const uint32_t *key = nullptr;   // switching key (not for MODUP)
  int slot = 0;                    // workspace slot of this item
  int ext_slot = 0;                // MODDOWN / IPX: slot whose EXT holds the shared ModUp output
  int npoly = 2;                   // MDX: polynomials brought down (1 or 2)
};

struct Stage {
  // NTT1: both passes of a transform in one cluster launch (segs: the first pass's limbs
  // and prologue; segs2: the same limbs with the second pass's destination and epilogue)
  // IPN: the special limbs' inner product fused with ModDown's first inverse-NTT pass
  enum Kind { NTT, BCONV, IP, EW, FORK, JOIN_RECORD, JOIN_WAIT, NTT1, IPN } kind = NTT;
  bool column = false, fwd = false;
  int pro = 0, epi = 0, ewop = 0;
  bool aux = false;
  bool gather_own = false, gather_ext = false;
  bool add_c1 = false;  // IP: some item adds its pass-through polynomial to both halves
  int max_in = 0, max_out = 0;
  std::vector<fhe::Seg> segs;
  std::vector<fhe::Seg> segs2;
  std::vector<fhe::BconvGroup> groups;
};

struct Program {
  std::vector<fhe::KsArgs> ks;  // per item
  std::vector<Stage> stages;
};

// Device copies of a program's launch descriptors (for captured plans).
struct DevProgram {
  void *buf = nullptr;
  std::vector<fhe::SegList> lists;   // per stage (segment stages)
  std::vector<fhe::SegList> lists2;  // per stage (NTT1: the second pass's segments)
  std::vector<fhe::BconvArgs> bargs; // per stage (BConv stages)
};

int ensure_slots(fhe_ctx *c, int n);
int build_program(fhe_ctx *c, const std::vector<Item> &items, bool fused, Program &P);
bool program_fits_inline(const Program &P);
int run_program_inline(fhe_ctx *c, const Program &P, cudaStream_t s);
int upload_program(fhe_ctx *c, const Program &P, DevProgram &D);
// lane: which lane's auxiliary stream and fork / join events the program uses
int run_program_dev(fhe_ctx *c, const Program &P, const DevProgram &D, cudaStream_t s, int lane);
void free_program(DevProgram &D);
int run_items_chunked(fhe_ctx *c, const std::vector<Item> &items, int first_slot, cudaStream_t s);
