"""Generate tap_dispatch.cuh: the per-chunk tap loop of the sparse mixing kernel as inline PTX.

Each lane owns R consecutive outputs n .. n+R-1 and holds the register window
win[0 .. 2R) = lo ++ hi = y[n - (c+1)R .. n - cR + R) for the current chunk c of filter
offsets [cR, cR + R).  A tap of ear e at offset cR + delta with weight w needs

    acc_e[r] += w * win[R - delta + r]      for r = 0 .. R-1

with a fixed window register for every (delta, r).  TapChunk<R>::run applies all taps of
one chunk: it walks the chunk's tap list in shared memory (entries {code, weight bits},
code = delta + R * e, warp-uniform), and for each tap one indirect branch (brx.idx.uni over
a .branchtargets table of the 2R straight-line FMA blocks) selects the block; the next
entry is loaded while the current block runs.  The whole loop is one asm statement, so the
window and accumulator registers are bound once per chunk.

Run:  python gen_tap_dispatch.py   (rewrites tap_dispatch.cuh next to this file).
"""
import os

R_VALUES = (12, 20, 28, 36, 44)


def gen(R: int) -> str:
    # operands: accL 0..R-1, accR R..2R-1, lo 2R..3R-1, hi 3R..4R-1, taps addr 4R, count 4R+1
    accL = lambda r: f"%{r}"
    accR = lambda r: f"%{R + r}"
    lo = lambda j: f"%{2 * R + j}"
    hi = lambda j: f"%{3 * R + j}"
    addr = f"%{4 * R}"
    count = f"%{4 * R + 1}"
    labels = [f"L{e}_{d}" for e in range(2) for d in range(R)]
    lines = [
        "{",
        ".reg .pred Pm;",
        ".reg .b32 Rc, Rcn, Rwn;",
        ".reg .f32 Rw;",
        ".reg .u32 Rp, Re;",
        "Ltab: .branchtargets " + ", ".join(labels) + ";",
        f"mov.u32 Rp, {addr};",
        f"mad.lo.u32 Re, {count}, 8, Rp;",
        "ld.shared.v2.b32 {Rcn, Rwn}, [Rp];",
        "Lloop:",
        "mov.b32 Rc, Rcn;",
        "mov.b32 Rw, Rwn;",
        "add.u32 Rp, Rp, 8;",
        "setp.lt.u32 Pm, Rp, Re;",
        "@Pm ld.shared.v2.b32 {Rcn, Rwn}, [Rp];",
        "brx.idx.uni Rc, Ltab;",
    ]
    for e in range(2):
        acc = accL if e == 0 else accR
        for d in range(R):
            lines.append(f"L{e}_{d}:")
            for r in range(R):
                j = R - d + r
                src = lo(j) if j < R else hi(j - R)
                lines.append(f"fma.rn.f32 {acc(r)}, Rw, {src}, {acc(r)};")
            lines.append("@Pm bra.uni Lloop;")
            lines.append("bra.uni Ldone;")
    lines += ["Ldone:", "}"]
    body = "\n".join('        "' + ln + '\\n"' for ln in lines)
    outs = ", ".join([f'"+f"(accL[{r}])' for r in range(R)] + [f'"+f"(accR[{r}])' for r in range(R)])
    ins = ", ".join([f'"f"(lo[{r}])' for r in range(R)] + [f'"f"(hi[{r}])' for r in range(R)] +
                    ['"r"(taps)', '"r"(n)'])
    return f"""template <>
struct TapChunk<{R}> {{
    // taps: shared-memory address of n >= 1 entries {{code, weight bits}}
    static __device__ __forceinline__ void run(const float (&lo)[{R}], const float (&hi)[{R}],
                                               float (&accL)[{R}], float (&accR)[{R}],
                                               uint32_t taps, int n)
    {{
        asm volatile(
{body}
        : {outs}
        : {ins}
        : "memory");
    }}
}};
"""


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    parts = ["// tap_dispatch.cuh -- GENERATED by gen_tap_dispatch.py; do not edit by hand.",
             "//",
             "// TapChunk<R>::run(lo, hi, accL, accR, taps, n): all n taps of one filter chunk of the",
             "// sparse mixing kernel, acc_e[r] += w * (lo ++ hi)[R - delta + r] for r < R, one",
             "// brx.idx.uni jump per tap into straight-line FMA blocks (see gen_tap_dispatch.py).",
             "#pragma once", "", "#include <cstdint>", "", "namespace hrir {", "",
             "template <int R>", "struct TapChunk;", ""]
    for R in R_VALUES:
        parts.append(gen(R))
    parts.append("}  // namespace hrir\n")
    with open(os.path.join(here, "tap_dispatch.cuh"), "w") as f:
        f.write("\n".join(parts))


if __name__ == "__main__":
    main()
