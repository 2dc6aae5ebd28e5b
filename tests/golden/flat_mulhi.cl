__kernel void mulhi_flat(__global const uint *a, __global int *b)
{
    uint var0;
    var0 = a[get_local_id(0)];
    b[get_local_id(0)] = (int)(mul_hi((16702650u & 16777215u), (var0 & 16777215u)) + (uint)mul_hi(((int)(8388609u << 8) >> 8), ((int)(var0 << 8) >> 8)));
}
