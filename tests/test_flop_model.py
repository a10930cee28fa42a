"""The algorithmic FLOP model of bench.py (FP64 flops per accepted step, rejected attempt,
propagated measurement and track, counted from the kernel source) against hardware counts:
for every ncu capture kept in bench.CAPTURES, the model evaluated on the captured launch's unit
counts reproduces the model count recorded with it, and the executed FP64 flops the hardware
counted (2 dfma + dadd + dmul) lie between the model and 1.25 times it. The model counts a
division, square root or logarithm as one flop, while the hardware executes each as a sequence
of FP64 instructions, so executed >= model; a model that counted work the kernel does not do,
or a table entry changed without a new capture, fails here."""

import bench


def model_flops(variant: str, cap: dict, table=None) -> int:
    fa, fr, fh, ft = (table or bench.FLOPS)[variant]
    return (fa * (cap["attempts"] - cap["rejected"]) + fr * cap["rejected"] + fh * cap["hits_after_first"] +
            ft * cap["tracks"])


def test_model_reproduces_the_recorded_counts():
    for (workload, variant, regs), cap in bench.CAPTURES.items():
        table = bench.FLOPS_MAP if workload == "map" else bench.FLOPS
        assert model_flops(variant, cap, table) == cap["fp64_model"], (workload, variant, regs)


def test_executed_fp64_flops_bound_the_model():
    for key, cap in bench.CAPTURES.items():
        ratio = cap["fp64_exec"] / cap["fp64_model"]
        assert 1.0 <= ratio <= 1.25, (key, ratio)


def test_mixed_path_moves_the_stepping_off_the_fp64_pipe():
    # per accepted step the mixed path keeps only its FP64 anchors; per measurement the update
    # and the smoother stay FP64 (their count is at least the FP64 path's update + smoother part)
    fa64, fr64, fh64, _ = bench.FLOPS["fp64"]
    fam, frm, fhm, _ = bench.FLOPS["mixed"]
    assert fam < fa64 / 10 and frm < fr64 / 10
    assert 0.4 * fh64 < fhm < fh64
    # and the FP32 pipe carries the propagation instead: two orders of magnitude more FP32 flops
    cm, c64 = bench.CAPTURES[("barrel", "mixed", 128)], bench.CAPTURES[("barrel", "fp64", 128)]
    assert cm["fp32_exec"] > 50 * c64["fp32_exec"]
