"""Copy engine as plain memcpy -- TEST INFRASTRUCTURE ONLY.

The data plane moves (buffer, offset, len) regions between live device
memory, a device staging area and the pinned host image (Section 4.2 CoW
copies, Section 4.3 recopy, Section 5 chunked copies, Section 6 restore).
Here every descriptor is one numpy slice assignment (a memcpy).

Descriptor fields (one row per copy): src_off, dst_off, len, buf, flags.
  flags & 0xff = direction:
      1 live -> staging      2 live -> image
      3 staging -> image     4 image -> live
  flags & 0x100 = after the bytes land, set bit ``buf`` of the present bitmap
A live endpoint is addressed as (buffer index, offset inside the buffer) and
must satisfy off + len <= size[buf]; staging / image offsets must satisfy
off + len <= the area's byte size.  A descriptor that breaks a rule moves no
bytes and makes the call report EINVAL (1); the others are still applied.

Parity: pinned by tests against independent slicing over random regions,
including every offset 0..15 x length 0..300 combination.
"""
import numpy as np

LIVE_TO_STAGING, LIVE_TO_IMAGE, STAGING_TO_IMAGE, IMAGE_TO_LIVE = 1, 2, 3, 4
MARK_PRESENT = 0x100

DESC_DTYPE = np.dtype([("src_off", "<u8"), ("dst_off", "<u8"), ("len", "<u8"),
                       ("buf", "<u4"), ("flags", "<u4")])


def apply(desc, live, buf_off, buf_size, staging=None, image=None, present=None):
    """Apply descriptors in order.  live: uint8 arena; buf_off/buf_size:
    arena offset and size of each table buffer.  Returns 0 or 1 (EINVAL)."""
    err = 0
    n = len(buf_off)
    for d in desc:
        so, do, ln = int(d["src_off"]), int(d["dst_off"]), int(d["len"])
        b, fl = int(d["buf"]), int(d["flags"])
        kind = fl & 0xFF
        if fl & ~0x1FF or kind not in (1, 2, 3, 4):
            err = 1
            continue

        def live_ok(off):
            return b < n and off <= int(buf_size[b]) and ln <= int(buf_size[b]) - off

        def area_ok(area, off):
            return area is not None and off <= area.size and ln <= area.size - off

        if kind == LIVE_TO_STAGING:
            ok = live_ok(so) and area_ok(staging, do)
        elif kind == LIVE_TO_IMAGE:
            ok = live_ok(so) and area_ok(image, do)
        elif kind == STAGING_TO_IMAGE:
            ok = area_ok(staging, so) and area_ok(image, do)
        else:
            ok = area_ok(image, so) and live_ok(do)
        if (fl & MARK_PRESENT) and (present is None or b >= n):
            ok = False
        if not ok:
            err = 1
            continue
        if kind == LIVE_TO_STAGING:
            a = int(buf_off[b]) + so
            staging[do:do + ln] = live[a:a + ln]
        elif kind == LIVE_TO_IMAGE:
            a = int(buf_off[b]) + so
            image[do:do + ln] = live[a:a + ln]
        elif kind == STAGING_TO_IMAGE:
            image[do:do + ln] = staging[so:so + ln]
        else:
            a = int(buf_off[b]) + do
            live[a:a + ln] = image[so:so + ln]
        if fl & MARK_PRESENT:
            present[b >> 5] |= np.uint32(1 << (b & 31))
    return err
