"""ctypes binding of libigs_peaks.so (include/igs_peaks.h): throughput probes
for the roofline's denominators. Measurement only; the rasteriser does not
use it."""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libigs_peaks.so")
KINDS = {"ffma": 0, "ffma2": 1, "ex2": 2, "fmnmx": 3, "fmnmx3": 4, "imnmx": 5, "match": 6}

_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2407_01866_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        lib.igs_peak_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_float)]
        lib.igs_peak_probe.restype = ctypes.c_int
        _lib = lib
    return _lib


def probe(kind, iters=2000, reps=5):
    """Runs one probe on the current device: returns (lane-ops/s,
    instructions/s, fastest launch in ms)."""
    o, i, ms = ctypes.c_double(), ctypes.c_double(), ctypes.c_float()
    rc = load().igs_peak_probe(KINDS[kind], iters, reps, ctypes.byref(o), ctypes.byref(i),
                               ctypes.byref(ms))
    if rc != 0:
        raise RuntimeError(f"igs_peak_probe({kind}) failed with {rc}")
    return o.value, i.value, ms.value


def main():
    """Prints every probe's rates on the current device as one JSON line:
    python -m paper_2407_01866_b300.peaks"""
    import json
    out = {}
    for kind in KINDS:
        iters = 200 if kind == "match" else 2000
        ops, inst, ms = probe(kind, iters=iters, reps=5)
        out[kind] = {"lane_ops_per_s": ops, "instructions_per_s": inst, "best_ms": ms}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
