__kernel void lds_swap(__global int *a, __local int *tmp)
{
    int var0;
    int var1;
    var0 = a[get_local_id(0)];
    tmp[get_local_id(0)] = var0;
    barrier(CLK_LOCAL_MEM_FENCE);
    var1 = tmp[(63u & (1u + get_local_id(0)))];
    a[get_local_id(0)] = (int)((uint)var1 + (uint)var0);
}
