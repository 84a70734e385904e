"""Measured peaks of the FP64 FMA, FP32 FMA and packed FP32x2 FMA pipes
(``csrc_peaks/fei_peaks.cu``), the denominators of the CUDA-core rooflines.

``measure()`` times each probe with CUDA events on the current stream: one
calibration launch, then launches of about ``target_ms`` each, best of
``reps``; every launch fills the GPU with 8 blocks of 256 threads per SM.
Returns TFLOP/s per pipe.  The bf16/fp16 tensor peak and the HBM copy
bandwidth come from the driver's MEASURED_PEAKS.json; the TF32 tensor peak
is measured here with a library GEMM (torch.matmul of FP32 operands with
TF32 allowed), as the driver measures bf16.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfei_peaks.so")

KINDS = {"fp64_fma": 0, "fp32_fma": 1, "fp32x2_fma": 2}


def _lib():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built (paper_1310_1194_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    lib.fei_peak_probe_launch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p]
    lib.fei_peak_probe_launch.restype = ctypes.c_double
    return lib


def measure(target_ms: float = 40.0, reps: int = 5) -> dict:
    import torch
    lib = _lib()
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    res = {"blocks": blocks, "threads_per_block": 256, "chains_per_thread": 8, "reps": reps}

    def timed(kind, iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = lib.fei_peak_probe_launch(kind, blocks, iters, ctypes.c_void_p(out.data_ptr()), sp)
        e1.record(stream)
        e1.synchronize()
        if flops < 0:
            raise RuntimeError(f"peak probe {kind} failed to launch")
        return flops, e0.elapsed_time(e1)

    for name, kind in KINDS.items():
        it = 2000
        _, ms = timed(kind, it)
        it = max(1, int(it * target_ms / max(ms, 1e-3)))
        best = 0.0
        for _ in range(reps):
            flops, ms = timed(kind, it)
            best = max(best, flops / (ms * 1e-3) / 1e12)
        res[name + "_tflops"] = best
        res[name + "_iters"] = it
    # TF32 tensor peak (library GEMM), 8192^3, best of reps
    a = torch.randn(8192, 8192, device="cuda")
    b = torch.randn(8192, 8192, device="cuda")
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        torch.matmul(a, b)
        best = 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.matmul(a, b)
            e1.record(stream)
            e1.synchronize()
            best = max(best, 2 * 8192 ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        res["tf32_tensor_tflops"] = best
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    del a, b, out
    return res


if __name__ == "__main__":
    import json
    print(json.dumps(measure(), indent=1))
