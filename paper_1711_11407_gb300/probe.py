"""Random-gather ceiling of this GPU: python -m paper_1711_11407_gb300.probe [log2_elems] [reps]

Times fpssft_probe_gather (random 8-byte reads over a buffer much larger than L2) for both load
flavours, single and adjacent-pair accesses, with CUDA events, and prints one JSON line per case."""
import json
import sys

import torch

from .api import probe_gather


def measure(log2_elems=29, reps=5, threads_total=152 * 16 * 256, reads=64):
    buf = torch.zeros(1 << log2_elems, dtype=torch.complex64, device="cuda")
    out = []
    for load_mode in (0, 1):
        for pair in (0, 1):
            probe_gather(buf, reads, threads_total, load_mode, pair)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                probe_gather(buf, reads, threads_total, load_mode, pair)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            acc = threads_total * reads
            out.append({"load_mode": ["ld.global.nc", "ld.global.cg"][load_mode], "pair": pair, "ms": ms,
                        "accesses_per_s": acc / ms * 1e3, "useful_GBs": acc * 8 * (1 + pair) / ms / 1e6,
                        "buffer_bytes": buf.numel() * 8})
    return out


if __name__ == "__main__":
    a = sys.argv[1:]
    for row in measure(int(a[0]) if a else 29, int(a[1]) if len(a) > 1 else 5):
        print(json.dumps(row))
