"""Summarise ncu output (one-kernel raw export, or a launch list) as short text.

  python -m paper_1611_04474_gb300.ncu_summary raw  <ncu --page raw --csv export>
  python -m paper_1611_04474_gb300.ncu_summary list <ncu --csv launch list>
"""
import csv
import sys
from collections import OrderedDict

RAW_KEYS = [
    "gpu__time_duration.sum",
    "smsp__inst_executed.sum",
    "smsp__issue_active.avg.pct_of_peak_sustained_active",
    "sm__warps_active.avg.pct_of_peak_sustained_active",
    "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_fma.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active",
    "smsp__inst_executed_op_shared_atom.sum",
    "l1tex__data_pipe_lsu_wavefronts_mem_shared_op_ld.sum",
    "l1tex__data_bank_conflicts_pipe_lsu_mem_shared_op_ld.sum",
    "dram__bytes_read.sum",
    "dram__bytes_write.sum",
    "lts__t_bytes.sum",
    "launch__registers_per_thread",
    "launch__shared_mem_per_block_static",
    "launch__shared_mem_per_block_dynamic",
    "launch__occupancy_limit_registers",
    "launch__occupancy_limit_shared_mem",
    "launch__grid_size",
]


def raw(path):
    rows = list(csv.reader(open(path)))
    hdr, units = rows[0], rows[1]
    for r in rows[2:]:
        d = {h: (v, u) for h, v, u in zip(hdr, r, units)}
        print(f"kernel: {d.get('Kernel Name', ('?',))[0][:100]}")
        for k in RAW_KEYS:
            if k in d:
                print(f"  {k:62s} {d[k][0]:>16s} {d[k][1]}")
        st = []
        for k in hdr:
            if k.startswith("smsp__pcsamp_warps_issue_stalled_") and not k.endswith("not_issued"):
                try:
                    st.append((k[len("smsp__pcsamp_warps_issue_stalled_"):], float(d[k][0].replace(",", ""))))
                except ValueError:
                    pass
        tot = sum(v for _, v in st) or 1.0
        st.sort(key=lambda x: -x[1])
        print("  stall samples: " + ", ".join(f"{k} {100 * v / tot:.0f}%" for k, v in st[:8]))


def launch_list(path):
    rows = [r for r in csv.reader(open(path)) if len(r) > 10]
    hdr = rows[0]
    ki, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    agg = OrderedDict()
    for r in rows[1:]:
        name = r[ki].split("(")[0][:70]
        scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}.get(r[ui], 1.0)
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += float(r[vi].replace(",", "")) * scale
    tot = sum(v[1] for v in agg.values())
    print(f"{'kernel':70s} {'launches':>8s} {'total us':>12s} {'share':>7s}")
    for k, (c, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"{k:70s} {c:8d} {t:12.1f} {100 * t / tot:6.1f}%")


if __name__ == "__main__":
    {"raw": raw, "list": launch_list}[sys.argv[1]](sys.argv[2])
