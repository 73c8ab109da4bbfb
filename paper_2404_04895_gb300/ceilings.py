"""Roofline ceilings of the construction step, measured on the current GPU
with the library's measurement kernels (aco_ceiling_*), timed with CUDA
events on the launching stream:

  row_reads  bytes/s for whole random rows of an M_p-sized buffer read with
             16-byte coalesced loads -- the full-scan construction's traffic
             (rows of n = 5000 fp32 / bf16 entries from 100 MB / 50 MB
             buffers, which the L2 holds, and from 1 GB, which it cannot)
  philox     scored candidates/s: Philox4x32-10 blocks, four candidates
             each, fl32(r * p) and a running argmax -- the scan's arithmetic
  chase      clock cycles per dependent load through a 100 MB buffer -- the
             latency a construction step waits when its next row is not
             already in flight

  python -m paper_2404_04895_gb300.ceilings        (prints one JSON object)
"""
import json

import numpy as np

MB = 1 << 20


def _time(torch, stream, fn, reps, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def measure(reps=5, chase=True):
    import torch

    from . import binding as B
    B.lib()
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    st = torch.cuda.current_stream()
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = {"sms": sms, "reps": reps, "statistic": "best of reps launches after 2 warm-ups"}

    rows = []
    warps = sms * 64
    for footprint, row_bytes, what in [(100 * MB, 20000, "fp32 M_p, n = 5000"),
                                       (50 * MB, 10000, "bf16 M_p, n = 5000"),
                                       (1024 * MB, 20000, "1 GB: beyond the L2")]:
        buf = torch.ones(footprint // 4, dtype=torch.int32, device="cuda")
        rpw = 8
        salt = [0]

        def go():
            salt[0] += 1
            B.ceiling_row_reads(buf, footprint, row_bytes, warps, rpw, salt[0], sink, st)

        ms = _time(torch, st, go, reps)
        nbytes = warps * rpw * row_bytes
        rows.append({"footprint_MB": footprint // MB, "row_bytes": row_bytes, "what": what,
                     "bytes_per_launch": nbytes, "ms": round(ms, 4), "GBps": round(nbytes / (ms / 1e3) / 1e9, 1)})
        del buf
    out["row_reads"] = rows

    threads, bpt = sms * 2048, 256
    salt = [0]

    def ph():
        salt[0] += 1
        B.ceiling_philox(0, threads, bpt, salt[0], sink, st)

    ms = _time(torch, st, ph, reps)
    cands = 4 * threads * bpt
    out["philox"] = {"threads": threads, "blocks_per_thread": bpt, "candidates_per_launch": cands,
                     "ms": round(ms, 4), "candidates_per_s": round(cands / (ms / 1e3), 1)}

    if chase:
        slots = 100 * MB // 4
        rng = np.random.default_rng(1)
        perm = rng.permutation(slots).astype(np.uint32)
        nxt = np.empty(slots, dtype=np.uint32)
        nxt[perm] = np.roll(perm, -1)          # one cycle through every slot
        nd = torch.from_numpy(nxt).cuda()
        chains, hops = sms, 2048
        cyc = torch.zeros(chains, dtype=torch.int64, device="cuda")
        B.ceiling_chase(nd, slots, chains, hops, cyc, sink, st)     # warm the buffer into the L2
        B.ceiling_chase(nd, slots, chains, hops, cyc, sink, st)
        torch.cuda.synchronize()
        c = cyc.cpu().numpy()
        out["chase"] = {"footprint_MB": 100, "chains": chains, "hops": hops,
                        "cycles_per_load_median": float(np.median(c)), "cycles_per_load_min": int(c.min()),
                        "cycles_per_load_max": int(c.max())}
    return out


if __name__ == "__main__":
    print(json.dumps(measure()))
