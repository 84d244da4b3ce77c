"""Instruction issue rates of the GPU, the denominators of the library's integer rooflines.

The cost kernels' roofline counts masked 32-bit popcounts (POPC per clock), the describe roofline
counts 32-bit integer lane operations (the ALU pipe's lanes per clock). `measure()` runs the probe
in libbsm_probe.so (probe/issue_rate.cu) once per instruction; `write_summary()` records the result
as a short text summary with the probe source's hash; `load()` reads that summary back, and only if
the probe source is unchanged since it was written.

  python -m paper_1402_2020_gb300.peaks [--write PATH]
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import re
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
PROBE_SRC = os.path.join(HERE, "probe", "issue_rate.cu")
PROBE_LIB = os.path.join(HERE, "_lib", "libbsm_probe.so")
SUMMARY = os.path.join(os.path.dirname(HERE), "profiles", "int_issue_rates_gb300.md")

# op index in the probe -> name (the SASS-level instruction each inline-PTX form issues; MIN16X2_LOP3 is a
# packed 16-bit minimum followed by a LOP3, counted as one step)
OPS = ("POPC", "LOP3", "IADD", "SHF", "PRMT", "IMAD", "VABSDIFF4", "DP4A", "IMNMX", "SHFL", "REDUX", "FFMA",
       "HFMA2", "MIN16X2_LOP3")


def source_hash() -> str:
    with open(PROBE_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measure(ctas_per_sm: int = 8, iters: int = 4096) -> dict:
    """{name: lanes per clock per SM} plus "_sm_mhz" (median SM clock seen by the probe)."""
    if not os.path.exists(PROBE_LIB):
        raise ImportError(f"libbsm_probe.so is not built ({PROBE_LIB}); run __graft_entry__.build() first")
    L = ctypes.CDLL(PROBE_LIB)
    L.bsm_probe_issue_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
    L.bsm_probe_issue_rate.restype = ctypes.c_int
    assert L.bsm_probe_op_count() == len(OPS)
    out, mhz = {}, []
    for i, name in enumerate(OPS):
        r, m = ctypes.c_double(), ctypes.c_double()
        st = L.bsm_probe_issue_rate(i, ctas_per_sm, iters, ctypes.byref(r), ctypes.byref(m))
        if st != 0:
            raise RuntimeError(f"issue-rate probe of {name} failed with CUDA error {st}")
        out[name] = r.value
        mhz.append(m.value)
    out["_sm_mhz"] = sorted(mhz)[len(mhz) // 2]
    return out


def write_summary(rates: dict, path: str = SUMMARY, gpu: str = "", command: str = "") -> None:
    lines = [
        "# Instruction issue rates on the GB300 (lanes per clock per SM)",
        "",
        "Measured by `probe/issue_rate.cu` (built into `paper_1402_2020_gb300/_lib/libbsm_probe.so`): one kernel per",
        "instruction, eight 256-thread CTAs per SM, eight independent dependency chains of the instruction per",
        "thread in inline PTX, 4096 x 32 instructions per thread; per SM the lane-instructions its CTAs retired",
        "over the span of their clock64 readings, median over the SMs.",
        "",
        f"Command: `{command or 'python -m paper_1402_2020_gb300.peaks --write profiles/int_issue_rates_gb300.md'}`",
        f"GPU: {gpu or 'NVIDIA GB300'}; SM clock during the probe (clock64 over the global timer, median): "
        f"{rates['_sm_mhz']:.0f} MHz",
        "",
        "| instruction | lanes / clk / SM |",
        "|---|---|",
    ]
    lines += [f"| {n} | {rates[n]:.2f} |" for n in OPS]
    lines += ["", "Machine-readable lines (bench.py reads these while the probe source is unchanged):", ""]
    lines += [f"issue_rate: {n} {rates[n]:.3f} source_sha256={source_hash()}" for n in OPS]
    lines += [f"probe_sm_mhz: {rates['_sm_mhz']:.1f} source_sha256={source_hash()}", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))


def load(path: str = SUMMARY) -> dict | None:
    """Rates recorded in the summary, or None if it is missing or was measured with another probe source."""
    try:
        text = open(path).read()
    except OSError:
        return None
    digest = source_hash()
    out = {}
    for line in text.splitlines():
        m = re.match(r"issue_rate:\s*(\w+)\s+([0-9.]+)\s+source_sha256=(\w+)", line.strip())
        if m and m.group(3) == digest:
            out[m.group(1)] = float(m.group(2))
        m = re.match(r"probe_sm_mhz:\s*([0-9.]+)\s+source_sha256=(\w+)", line.strip())
        if m and m.group(2) == digest:
            out["_sm_mhz"] = float(m.group(1))
    return out if all(n in out for n in OPS) else None


FP8_SUMMARY = os.path.join(os.path.dirname(HERE), "profiles", "fp8_gemm_gb300.md")


def measure_fp8_gemm(n: int = 8192, reps: int = 20) -> dict:
    """Dense E4M3 x E4M3 -> bf16 GEMM rate of the vendor library (cuBLASLt through torch._scaled_mm), n^3,
    best of `reps` single launches and the mean of `reps` back-to-back launches, in TFLOP/s."""
    import torch

    g = torch.Generator(device="cuda").manual_seed(7)
    a = (torch.rand((n, n), device="cuda", generator=g) - 0.5).to(torch.float8_e4m3fn)
    b = (torch.rand((n, n), device="cuda", generator=g) - 0.5).to(torch.float8_e4m3fn).t()  # column-major operand
    one = torch.ones((), device="cuda", dtype=torch.float32)

    def run():
        return torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)

    for _ in range(3):
        run()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    e1.synchronize()
    mean = e0.elapsed_time(e1) * 1e-3 / reps
    flops = 2.0 * n ** 3
    return {"n": n, "burst_tflops": flops / best / 1e12, "loop_tflops": flops / mean / 1e12}


def write_fp8_summary(r: dict, path: str = FP8_SUMMARY, gpu: str = "") -> None:
    lines = [
        "# Dense E4M3 GEMM rate on the GB300 (the tensor-core cost kernel's roofline denominator)",
        "",
        "Measured by `paper_1402_2020_gb300/peaks.py` (`measure_fp8_gemm`): torch._scaled_mm (cuBLASLt), E4M3 x E4M3 -> bf16,",
        f"unit scales, {r['n']}^3 (2 n^3 flops), CUDA events; best single launch (burst) and the mean of back-to-back launches.",
        "",
        "Command: `python -m paper_1402_2020_gb300.peaks --fp8 --write-fp8 profiles/fp8_gemm_gb300.md`",
        f"GPU: {gpu or 'NVIDIA GB300'}",
        "",
        "| quantity | TFLOP/s |",
        "|---|---|",
        f"| burst | {r['burst_tflops']:.1f} |",
        f"| back to back | {r['loop_tflops']:.1f} |",
        "",
        f"fp8_gemm_tflops: burst {r['burst_tflops']:.1f} loop {r['loop_tflops']:.1f}",
        "",
    ]
    with open(path, "w") as f:
        f.write("\n".join(lines))


def load_fp8(path: str = FP8_SUMMARY) -> dict | None:
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"fp8_gemm_tflops:\s*burst\s+([0-9.]+)\s+loop\s+([0-9.]+)", text)
    return {"burst_tflops": float(m.group(1)), "loop_tflops": float(m.group(2))} if m else None


def rounded(rates: dict, name: str) -> float:
    """The issue rate as a whole number of lanes per clock (measurement noise removed)."""
    return float(round(rates[name]))


if __name__ == "__main__":
    if "--fp8" in sys.argv:
        r = measure_fp8_gemm()
        print(f"fp8 GEMM: burst {r['burst_tflops']:.1f} TFLOP/s, back to back {r['loop_tflops']:.1f} TFLOP/s")
        if "--write-fp8" in sys.argv:
            import torch

            i = sys.argv.index("--write-fp8")
            write_fp8_summary(r, sys.argv[i + 1] if i + 1 < len(sys.argv) else FP8_SUMMARY,
                              gpu=torch.cuda.get_device_name())
        sys.exit(0)
    rates = measure()
    gpu = ""
    try:
        import torch

        gpu = torch.cuda.get_device_name()
    except Exception:  # noqa: BLE001 - the name is informative only
        pass
    for n in OPS:
        print(f"{n:10s} {rates[n]:8.2f} lanes/clk/SM")
    print(f"SM clock {rates['_sm_mhz']:.0f} MHz")
    if "--write" in sys.argv:
        i = sys.argv.index("--write")
        write_summary(rates, sys.argv[i + 1] if i + 1 < len(sys.argv) else SUMMARY, gpu=gpu)
